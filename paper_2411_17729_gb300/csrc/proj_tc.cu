// proj_tc.cu -- the wide projections around the cascade on the tcgen05 tensor
// cores (BF16 split), for plans whose p and q are multiples of 16:
//
//   first stage fused with the input projection (§3, Eq. 3.2 with v^(0) = Bbar u):
//       v^(1)_l = Bbar u_l + (Abar Bbar) u_(l-1)      (second term on odd l only in
//                                                       the work-efficient schedule's
//                                                       first up-sweep level)
//   output projection (end of §3):           y_l = C v_l + D u_l
//   adjoint seed of the backward:            W_l = C^T G_l
//   adjoint of the first stage:              du_l = Bbar^T W_l + (Abar Bbar)^T W_(l+1) + D^T G_l
//
// Each is one sum of products over a 128-row tile of one sequence,
//
//     OUT[l, n] = sum_t sum_k A_t[l + d_t, k] B_t[n, k],     n in [n0, n0 + BN),
//
// with A_t time-major (u, G or state rows; K_t = p, q or m contiguous) and B_t
// the small matrix stored [N, K_t] (K contiguous): both are the K-major operands
// of tcgen05.mma, loaded by TMA in boxes of 32 K-entries (64 bytes, 64-byte
// swizzle; with K = 16 the box's upper half lies past the matrix and TMA fills
// it with zeros).  Every operand is a (hi, lo) BF16 pair and the product is
// taken as hi*hi + hi*lo + lo*hi with FP32 accumulation in TMEM, as in the
// stage kernel.  Rows whose source l + d_t lies outside the sequence read zero
// (x_(-1) = 0).  The epilogue writes FP32 rows (y, du: 16 columns per TMEM
// load) or (hi, lo) BF16 state rows (v^(1), W): each warp stages its 32 rows x
// 32 columns in a swizzled shared buffer (two per warp, alternating) and one
// TMA store per plane writes them as whole lines; a warp whose rows run past
// the sequence end stores its valid rows directly instead.
//
// Block layout (192 threads, persistent over (tile, column block)):
//   warp 0 TMA producer, warp 1 TMEM allocator + MMA issuer, warps 2..5 epilogue.
#include "common.cuh"
#include "ptx.cuh"

#include <algorithm>
#include <cstring>

namespace cascade {
namespace {

constexpr int BM = 128;                       // tile rows (M)
constexpr int KC = 32;                        // K entries per 64-byte operand row
constexpr int NTH = 192;
constexpr int MAXT = 3;                       // terms per projection
constexpr uint32_t ROWB = 64;
constexpr uint32_t A_BYTES = BM * ROWB;       // one plane of an A chunk: 8 KB

constexpr uint32_t OST_BYTES = 4096;          // one staging buffer: 32 rows x 64 B x 2 planes

struct ProjMaps {
  CUtensorMap a_hi[MAXT], a_lo[MAXT], b_hi[MAXT], b_lo[MAXT];
  CUtensorMap o_hi[2], o_lo[2];   // (hi, lo) output planes: [0] fixed buffer or buffer 0, [1] buffer 1
};

struct ProjArgs {
  const Tile* tiles;
  int32_t ntiles;
  int32_t N, BN, nblocks;
  int32_t nterms;
  int32_t K[MAXT];
  int32_t shift[MAXT];      // term t reads source row l + shift[t]
  int32_t odd_only;         // term 1 contributes on odd l only
  int32_t stages;
  float* out32;             // FP32 rows [rows, N], or null: (hi, lo) planes of `out`
  Bufs out;                 // buffer (tile.flags + 1) & 1 if buf_mode, else buf_fixed
  int32_t buf_mode, buf_fixed;
  int32_t* err;
  int32_t* diag;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ void raise_proj_timeout(const ProjArgs& a, volatile int* abort_flag,
                                                   int site, int x) {
  if (atomicCAS(a.err, 0, (int32_t)CASCADE_ERR_TIMEOUT) == 0 && a.diag) {
    a.diag[0] = 200 + site;
    a.diag[1] = (int32_t)blockIdx.x;
    a.diag[2] = x;
    a.diag[3] = 0;
    a.diag[4] = -1;
  }
  *abort_flag = 1;
}

// Row r of a tile reads zero in term t: its source lies outside the sequence,
// or (odd-only term) l is even.
__device__ __forceinline__ bool zero_row(const Tile& t, int r, int shift, bool odd) {
  const int src = t.t0 + r + shift;
  return src < 0 || (shift > 0 && src >= t.len) || (odd && ((t.t0 + r) & 1) == 0);
}

__global__ void __launch_bounds__(NTH, 1)
    proj_tc_kernel(const __grid_constant__ ProjMaps maps, const ProjArgs args) {
  const int BN = args.BN;
  const int S = args.stages;
  const int nwork = args.ntiles * args.nblocks;
  const uint32_t b_bytes = (uint32_t)BN * ROWB;
  const uint32_t stage_bytes = 2 * A_BYTES + 2 * b_bytes;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const bool split = args.out32 == nullptr;
  uint8_t* ostage = smem + (size_t)S * stage_bytes;         // 4 warps x 2 staging buffers
  uint64_t* full = reinterpret_cast<uint64_t*>(ostage + (split ? 8 * OST_BYTES : 0));
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tmem_cols = (2 * BN <= 32) ? 32u : (2 * BN <= 64) ? 64u : (2 * BN <= 128) ? 128u
                             : (2 * BN <= 256) ? 256u : 512u;

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
    for (int t = 0; t < args.nterms; ++t) {
      ptx::prefetch_tmap(&maps.a_hi[t]);
      ptx::prefetch_tmap(&maps.a_lo[t]);
      ptx::prefetch_tmap(&maps.b_hi[t]);
      ptx::prefetch_tmap(&maps.b_lo[t]);
    }
    if (split) {
      ptx::prefetch_tmap(&maps.o_hi[0]);
      ptx::prefetch_tmap(&maps.o_lo[0]);
      if (args.buf_mode) {
        ptx::prefetch_tmap(&maps.o_hi[1]);
        ptx::prefetch_tmap(&maps.o_lo[1]);
      }
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
  // launched as a programmatic dependent: the set-up above overlaps the
  // previous launch; nothing below runs before it has completed
  ptx::griddep_launch_dependents();
  ptx::griddep_wait();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued_parity[8];
      for (int s = 0; s < 8; ++s) issued_parity[s] = -1;
      bool ok = true;
      for (int w = blockIdx.x; w < nwork && ok && !*abort_flag; w += gridDim.x) {
        const Tile t = args.tiles[w / args.nblocks];
        const int n0 = (w % args.nblocks) * BN;
        const int row0 = (int)(t.seq_row0 + t.t0);
        const int brow = t.sys * args.N + n0;
        for (int tt = 0; tt < args.nterms && ok; ++tt) {
          // a source row before the tensor (row0 + shift = -1) is a negative TMA
          // coordinate: the load fills zeros there
          const int arow = row0 + args.shift[tt];
          for (int c = 0; c < (args.K[tt] + KC - 1) / KC; ++c) {
            if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag)) {
              raise_proj_timeout(args, abort_flag, 1, w);
              ok = false;
              break;
            }
            uint8_t* sa = smem + (size_t)stage * stage_bytes;
            ptx::mbar_arrive_expect_tx(&full[stage], stage_bytes);
            ptx::tma_load_2d(sa, &maps.a_hi[tt], &full[stage], c * KC, arow);
            ptx::tma_load_2d(sa + A_BYTES, &maps.a_lo[tt], &full[stage], c * KC, arow);
            ptx::tma_load_2d(sa + 2 * A_BYTES, &maps.b_hi[tt], &full[stage], c * KC, brow);
            ptx::tma_load_2d(sa + 2 * A_BYTES + b_bytes, &maps.b_lo[tt], &full[stage], c * KC,
                             brow);
            issued_parity[stage] = (int)phase;
            if (++stage == S) { stage = 0; phase ^= 1u; }
          }
        }
      }
      // never leave the block with copies in flight
      for (int s = 0; s < S; ++s)
        if (issued_parity[s] >= 0) ptx::mbar_wait(&full[s], (uint32_t)issued_parity[s], limit, nullptr);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = ptx::make_idesc(1u, BM, BN);
    int stage = 0;
    uint32_t phase = 0;
    int acc_i = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < nwork && ok && !*abort_flag; w += gridDim.x) {
      const Tile t = args.tiles[w / args.nblocks];
      const int abuf = acc_i & 1;
      const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&acc_empty[abuf], aph ^ 1u, limit, abort_flag))) {
        raise_proj_timeout(args, abort_flag, 2, w);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * BN);
      bool first = true;
      for (int tt = 0; tt < args.nterms && ok; ++tt) {
        const int sh = args.shift[tt];
        const bool odd = args.odd_only && tt == 1;
        const bool zeros = odd || t.t0 + sh < 0 || (sh > 0 && t.t0 + BM + sh > t.len);
        for (int c = 0; c < (args.K[tt] + KC - 1) / KC; ++c) {
          if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[stage], phase, limit, abort_flag))) {
            raise_proj_timeout(args, abort_flag, 3, w);
            ok = false;
            break;
          }
          uint8_t* sa = smem + (size_t)stage * stage_bytes;
          if (zeros) {
            // row r occupies bytes [64 r, 64 r + 64) of each A plane (the swizzle
            // permutes 16-byte units within the row)
            uint4* zh = reinterpret_cast<uint4*>(sa);
            uint4* zl = reinterpret_cast<uint4*>(sa + A_BYTES);
            const uint4 z = make_uint4(0, 0, 0, 0);
            for (int i = lane; i < BM * 4; i += 32)
              if (zero_row(t, i >> 2, sh, odd)) { zh[i] = z; zl[i] = z; }
            ptx::fence_proxy_async_smem();
            __syncwarp();
          }
          ptx::tc_fence_after();
          if (lane == 0) {
            const uint64_t dah = ptx::make_sdesc_sw64(ptx::smem_addr(sa));
            const uint64_t dal = ptx::make_sdesc_sw64(ptx::smem_addr(sa + A_BYTES));
            const uint64_t dbh = ptx::make_sdesc_sw64(ptx::smem_addr(sa + 2 * A_BYTES));
            const uint64_t dbl = ptx::make_sdesc_sw64(ptx::smem_addr(sa + 2 * A_BYTES + b_bytes));
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint64_t adv = (uint64_t)kk * 2;   // 32 bytes per K = 16 step
              ptx::mma_bf16(d_tmem, dah + adv, dbh + adv, idesc, (first && kk == 0) ? 0u : 1u);
              ptx::mma_bf16(d_tmem, dah + adv, dbl + adv, idesc, 1u);
              ptx::mma_bf16(d_tmem, dal + adv, dbh + adv, idesc, 1u);
            }
            ptx::tc_commit(&empty[stage]);
          }
          __syncwarp();
          first = false;
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) break;
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
    const int quad = warp & 3;                 // TMEM lane quadrant of this warp
    const int r = quad * 32 + lane;            // tile row == TMEM lane
    uint8_t* obuf = ostage + (size_t)(warp - 2) * 2 * OST_BYTES;
    uint32_t nst = 0;                          // staged stores issued by this warp
    int acc_i = 0;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
      const Tile t = args.tiles[w / args.nblocks];
      const int n0 = (w % args.nblocks) * BN;
      const int abuf = acc_i & 1;
      const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&acc_full[abuf], aph, limit, abort_flag))) {
        raise_proj_timeout(args, abort_flag, 4, w);
        break;
      }
      ptx::tc_fence_after();
      const bool valid = t.t0 + r < t.len;
      const int64_t grow = t.seq_row0 + t.t0 + r;
      const int64_t o0 = grow * (int64_t)args.N + n0;
      const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(abuf * BN);
      if (!split) {
        for (int cc = 0; cc < BN / 16; ++cc) {
          float v[16];
          ptx::tmem_ld16(trow + (uint32_t)(cc * 16), v);
          if (valid) {
            float4* o4 = reinterpret_cast<float4*>(args.out32 + o0 + cc * 16);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          }
          __syncwarp();   // converged for the next tcgen05.ld
        }
      } else {
        const int b = args.buf_mode ? ((t.flags + 1) & 1) : args.buf_fixed;
        const int slot = args.buf_mode ? b : 0;
        // all 32 rows of this warp inside the sequence: staged TMA stores
        const bool staged = t.t0 + quad * 32 + 32 <= t.len;
        const int yrow = (int)(t.seq_row0 + t.t0 + quad * 32);
        __nv_bfloat16* ohi = static_cast<__nv_bfloat16*>(args.out.hi(b));
        __nv_bfloat16* olo = static_cast<__nv_bfloat16*>(args.out.lo(b));
        for (int cc = 0; cc < BN / 32; ++cc) {
          float v[32];
          ptx::tmem_ld32(trow + (uint32_t)(cc * 32), v);
          uint4 hq[4], lq[4];
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
            hq[j] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            lq[j] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
          if (staged) {
            uint8_t* sb = obuf + (nst & 1) * OST_BYTES;
            // the store issued two chunks ago has finished reading this buffer
            if (lane == 0) ptx::bulk_wait_read1();
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              *reinterpret_cast<uint4*>(sb + ptx::sw64_offset(lane, j)) = hq[j];
              *reinterpret_cast<uint4*>(sb + OST_BYTES / 2 + ptx::sw64_offset(lane, j)) = lq[j];
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              ptx::tma_store_2d(&maps.o_hi[slot], sb, n0 + cc * 32, yrow);
              ptx::tma_store_2d(&maps.o_lo[slot], sb + OST_BYTES / 2, n0 + cc * 32, yrow);
              ptx::bulk_commit();
            }
            ++nst;
          } else if (valid) {
            uint4* h4 = reinterpret_cast<uint4*>(ohi + o0 + cc * 32);
            uint4* l4 = reinterpret_cast<uint4*>(olo + o0 + cc * 32);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              h4[j] = hq[j];
              l4[j] = lq[j];
            }
          }
          __syncwarp();   // converged for the next tcgen05.ld
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(&acc_empty[abuf]);
      ++acc_i;
    }
    if (lane == 0) ptx::bulk_wait0();          // staged stores complete before the block exits
    __syncwarp();
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, tmem_cols);
}

// FP32 -> (hi, lo) BF16 planes, hi = RN(x), lo = RN(x - hi); four per thread.
__global__ void split_rows_kernel(const float4* __restrict__ x, int64_t n4,
                                  uint2* __restrict__ hi, uint2* __restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = x[i];
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
    const __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
    hi[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
    lo[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&l0), *reinterpret_cast<const uint32_t*>(&l1));
  }
}

// Rows of w FP32 values -> rows of wp >= w BF16 (hi, lo) entries, zero past w.
__global__ void split_rows_pad_kernel(const float* __restrict__ x, int64_t rows, int w, int wp,
                                      __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ lo) {
  const int64_t n = rows * wp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / wp;
    const int j = (int)(e - r * wp);
    const float v = j < w ? x[r * w + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// out[s][i][j] = split(M[s * ss + i * si + j * sj]), i < R, j < C.
__global__ void split_coef_kernel(const float* __restrict__ M, int64_t ss, int64_t si, int64_t sj,
                                  int R, int C, int ns, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  const int64_t n = (int64_t)ns * R * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / ((int64_t)R * C), rem = e - s * R * C;
    const int i = (int)(rem / C), j = (int)(rem - (int64_t)i * C);
    const float x = M[s * ss + (int64_t)i * si + (int64_t)j * sj];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// Columns per block: N itself up to 256 (a multiple of 16), else the largest
// power of two from 256 down to 32 that divides N.
int block_cols(int N) {
  if (N <= 256) return N % 16 == 0 ? N : 0;
  for (int bn = 256; bn >= 32; bn >>= 1)
    if (N % bn == 0) return bn;
  return 0;
}

struct Term {
  const void* a_hi;
  const void* a_lo;
  int64_t a_rows;
  int K;
  int shift;
  int coef;        // PC_* matrix of the B operand
};

// out32 null: (hi, lo) BF16 output rows in buffer (tile.flags + 1) & 1 (buf_mode)
// or buf_fixed of `out`, whose planes hold out_rows rows of N entries (N a
// multiple of 32).
cudaError_t launch_proj_tc(const Plan& p, const Tile* tiles, int ntiles, int N, int nterms,
                           const Term* terms, int odd_only, float* out32, const Bufs& out,
                           int64_t out_rows, int buf_mode, int buf_fixed, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const int BN = block_cols(N);
  const bool split = out32 == nullptr;
  if (BN == 0 || (split && BN % 32 != 0)) {
    set_global_error("tensor-core projection: unsupported output width");
    return cudaErrorInvalidValue;
  }
  ProjMaps maps;
  memset(&maps, 0, sizeof(maps));
  ProjArgs a{};
  std::string err;
  if (split) {
    for (int i = 0; i < (buf_mode ? 2 : 1); ++i) {
      const int b = buf_mode ? i : buf_fixed;
      if (!encode_tmap_2d(&maps.o_hi[i], out.hi(b), 2, N, out_rows, 32, 32, &err, 64) ||
          !encode_tmap_2d(&maps.o_lo[i], out.lo(b), 2, N, out_rows, 32, 32, &err, 64)) {
        set_global_error("tensor map encode failed: " + err);
        return cudaErrorInvalidValue;
      }
    }
  }
  for (int t = 0; t < nterms; ++t) {
    const Term& tm = terms[t];
    const auto* bh = static_cast<const __nv_bfloat16*>(p.pc_hi) + p.pc_off[tm.coef];
    const auto* bl = static_cast<const __nv_bfloat16*>(p.pc_lo) + p.pc_off[tm.coef];
    const uint64_t brows = (uint64_t)p.d.nsys * N;
    if (!encode_tmap_2d(&maps.a_hi[t], tm.a_hi, 2, tm.K, tm.a_rows, KC, BM, &err, 64) ||
        !encode_tmap_2d(&maps.a_lo[t], tm.a_lo, 2, tm.K, tm.a_rows, KC, BM, &err, 64) ||
        !encode_tmap_2d(&maps.b_hi[t], bh, 2, tm.K, brows, KC, BN, &err, 64) ||
        !encode_tmap_2d(&maps.b_lo[t], bl, 2, tm.K, brows, KC, BN, &err, 64)) {
      set_global_error("tensor map encode failed: " + err);
      return cudaErrorInvalidValue;
    }
    a.K[t] = tm.K;
    a.shift[t] = tm.shift;
  }
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.N = N;
  a.BN = BN;
  a.nblocks = N / BN;
  a.nterms = nterms;
  a.odd_only = odd_only;
  const uint32_t stage_bytes = 2 * A_BYTES + 2 * (uint32_t)BN * ROWB;
  const uint32_t ost = split ? 8 * OST_BYTES : 0;
  a.stages = std::min<int>(8, (int)((200u * 1024u - ost) / stage_bytes));
  a.out32 = out32;
  a.out = out;
  a.buf_mode = buf_mode;
  a.buf_fixed = buf_fixed;
  a.err = p.err;
  a.diag = p.err + 1;
  a.timeout_ns = 2000000000ull;
  const size_t smem = 1024 + (size_t)a.stages * stage_bytes + ost + 8 * (2 * a.stages + 5) + 16;
  cudaError_t e = cudaFuncSetAttribute(proj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int nwork = ntiles * a.nblocks;
  const int grid = std::min(nwork, p.num_sms);
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
  e = cudaLaunchKernelEx(&cfg, proj_tc_kernel, maps, a);
  CASCADE_LAUNCHED();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool proj_tc_supported(const Plan& p) {
  return p.d.precision == CASCADE_BF16_SPLIT && tile_rows(p) == BM && p.d.m % 32 == 0 &&
         p.d.p % 16 == 0 && p.d.q % 16 == 0 && p.d.p > 0 && p.d.q > 0;
}

size_t proj_coef_elems(const Plan& p, int64_t off[PC_COUNT]) {
  const int64_t m = p.d.m, pp = p.d.p, q = p.d.q, ns = p.d.nsys;
  const int64_t sizes[PC_COUNT] = {m * pp, m * pp, q * m, q * pp, m * q, pp * m, pp * m, pp * q};
  int64_t o = 0;
  for (int i = 0; i < PC_COUNT; ++i) {
    off[i] = o;
    o += (ns * sizes[i] + 127) / 128 * 128;   // 256-byte aligned starts
  }
  return (size_t)o;
}

cudaError_t launch_proj_coef(const Plan& p, cudaStream_t st) {
  const int m = p.d.m, pp = p.d.p, q = p.d.q, ns = p.d.nsys;
  struct Src {
    const float* M;
    int64_t ss, si, sj;
    int R, C;
  };
  const int64_t mp = (int64_t)m * pp, qm = (int64_t)q * m, qp = (int64_t)q * pp;
  const Src src[PC_COUNT] = {
      {p.Bbar32, mp, pp, 1, m, pp},    // PC_B     Bbar      [m, p]
      {p.ABbar32, mp, pp, 1, m, pp},   // PC_AB    Abar Bbar [m, p]
      {p.C32, qm, m, 1, q, m},         // PC_C     C         [q, m]
      {p.D32, qp, pp, 1, q, pp},       // PC_D     D         [q, p]
      {p.C32, qm, 1, m, m, q},         // PC_CT    C^T       [m, q]
      {p.Bbar32, mp, 1, pp, pp, m},    // PC_BT    Bbar^T    [p, m]
      {p.ABbar32, mp, 1, pp, pp, m},   // PC_ABT   (Abar Bbar)^T
      {p.D32, qp, 1, pp, pp, q},       // PC_DT    D^T       [p, q]
  };
  for (int i = 0; i < PC_COUNT; ++i) {
    const int64_t n = (int64_t)ns * src[i].R * src[i].C;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    split_coef_kernel<<<blocks, 256, 0, st>>>(
        src[i].M, src[i].ss, src[i].si, src[i].sj, src[i].R, src[i].C, ns,
        static_cast<__nv_bfloat16*>(p.pc_hi) + p.pc_off[i],
        static_cast<__nv_bfloat16*>(p.pc_lo) + p.pc_off[i]);
    CASCADE_LAUNCHED();
  }
  return cudaGetLastError();
}

cudaError_t launch_split_rows(const float* x, int64_t rows, int w, int wp, void* hi, void* lo,
                              cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  if (w == wp && w % 4 == 0) {
    const int64_t n4 = rows * w / 4;
    const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 8192);
    split_rows_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(x), n4,
                                              static_cast<uint2*>(hi), static_cast<uint2*>(lo));
  } else {
    const int64_t n = rows * wp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
    split_rows_pad_kernel<<<blocks, 256, 0, st>>>(x, rows, w, wp,
                                                  static_cast<__nv_bfloat16*>(hi),
                                                  static_cast<__nv_bfloat16*>(lo));
  }
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_proj_tc_stage0(const Plan& p, const Bufs& U, const Bufs& V, int64_t v_rows,
                                  int buf, bool odd_only, cudaStream_t st, int tile0, int ntiles) {
  const Term t[2] = {{U.hi(0), U.lo(0), p.rows, p.d.p, 0, PC_B},
                     {U.hi(0), U.lo(0), p.rows, p.d.p, -1, PC_AB}};
  if (ntiles < 0) ntiles = p.n_stage0_tiles - tile0;
  return launch_proj_tc(p, p.d_stage0_tiles + tile0, ntiles, p.d.m, 2, t, odd_only ? 1 : 0,
                        nullptr, V, v_rows, 0, buf, st);
}

cudaError_t launch_proj_tc_output(const Plan& p, const Bufs& U, float* y, const Bufs& V,
                                  int64_t v_rows, cudaStream_t st, int tile0, int ntiles) {
  for (const auto& sg : p.out_segs) {
    const Term t[2] = {{V.hi(sg[0]), V.lo(sg[0]), v_rows, p.d.m, 0, PC_C},
                       {U.hi(0), U.lo(0), p.rows, p.d.p, 0, PC_D}};
    // (a tile range applies within the list of all output tiles)
    const int a = std::max(sg[1], tile0);
    const int b = ntiles < 0 ? sg[1] + sg[2] : std::min(sg[1] + sg[2], tile0 + ntiles);
    if (b <= a) continue;
    const cudaError_t e = launch_proj_tc(p, p.d_out_tiles + a, b - a, p.d.q, 2, t, 0, y, Bufs{}, 0,
                                         0, 0, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_proj_tc_adj_init(const Plan& p, const Bufs& Gp, const Bufs& W,
                                    cudaStream_t st) {
  const Term t[1] = {{Gp.hi(0), Gp.lo(0), p.rows, p.d.q, 0, PC_CT}};
  return launch_proj_tc(p, p.d_all_tiles, p.n_all_tiles, p.d.m, 1, t, 0, nullptr, W, p.rows, 1, 0,
                        st);
}

cudaError_t launch_proj_tc_du(const Plan& p, const Bufs& Gp, const Bufs& W, int wbuf, float* du,
                              cudaStream_t st) {
  const Term t[3] = {{W.hi(wbuf), W.lo(wbuf), p.rows, p.d.m, 0, PC_BT},
                     {W.hi(wbuf), W.lo(wbuf), p.rows, p.d.m, 1, PC_ABT},
                     {Gp.hi(0), Gp.lo(0), p.rows, p.d.q, 0, PC_DT}};
  return launch_proj_tc(p, p.d_all_tiles, p.n_all_tiles, p.d.p, 3, t, 0, du, Bufs{}, 0, 0, 0, st);
}

}  // namespace cascade
