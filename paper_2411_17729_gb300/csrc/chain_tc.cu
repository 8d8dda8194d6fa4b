// chain_tc.cu -- the adjoint of the squaring chain (end of §2: P_(k+1) = P_k P_k)
// on the tensor cores, for the BF16-split plans:
//
//   dP_k += dP_(k+1) P_k^T + P_k^T dP_(k+1)
//
// X = dP_(k+1) (FP32) is split into BF16 (hi, lo) planes twice, as X and as X^T.
// Then both products take the stage kernel's form, K-major A times K-major B:
//   X P_k^T      A = X      (rows i, K = l)   B = P_k    (rows j, K = l)
//   P_k^T X      A = P_k^T  (rows i, K = l)   B = X^T    (rows j, K = l)
// each as three BF16 products (hi hi, hi lo, lo hi) accumulated in FP32 in one
// TMEM accumulator; the epilogue adds the accumulator to dP_k.
// One block per (128-row block, BN-column block, system); TMA loads into an
// S-stage ring, one thread issues the MMAs, four warps drain TMEM.
#include "common.cuh"
#include "ptx.cuh"

namespace cascade {
namespace {

constexpr int CBM = 128;            // rows per block (TMEM lanes)
constexpr int CKC = 32;             // K elements per 64-byte operand row
constexpr int CSTAGES = 4;
constexpr uint32_t CA_BYTES = CBM * 64;   // one A plane of a stage

struct ChainArgs {
  int m, kmax1, k, BN;
  float* dP;            // [nsys][kmax1][m][m]
  int64_t kst;          // elements between systems in dP
  // split planes of the finished dP_k for the next level (X and X^T, hi and lo), or null
  __nv_bfloat16 *oxh, *oxl, *oth, *otl;
  int32_t* err;
  unsigned long long timeout_ns;
};

// X = dP_(k+1) -> (hi, lo) BF16 planes of X and of X^T, [nsys * m, m] each.
__global__ void chain_split_kernel(const float* __restrict__ dPn, int64_t kst, int m,
                                   __nv_bfloat16* __restrict__ xh, __nv_bfloat16* __restrict__ xl,
                                   __nv_bfloat16* __restrict__ th, __nv_bfloat16* __restrict__ tl) {
  __shared__ float tile[32][33];
  const int s = blockIdx.z;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const float* X = dPn + (int64_t)s * kst;
  const int64_t base = (int64_t)s * m * m;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int i = i0 + yy, j = j0 + threadIdx.x;
    const float v = X[(int64_t)i * m + j];
    tile[yy][threadIdx.x] = v;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    xh[base + (int64_t)i * m + j] = h;
    xl[base + (int64_t)i * m + j] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int j = j0 + yy, i = i0 + threadIdx.x;      // X^T[j][i] = X[i][j]
    const float v = tile[threadIdx.x][yy];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    th[base + (int64_t)j * m + i] = h;
    tl[base + (int64_t)j * m + i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

__device__ __forceinline__ void chain_fail(const ChainArgs& a, volatile int* abort_flag, int site) {
  atomicCAS(a.err, 0, (int32_t)CASCADE_ERR_TIMEOUT);
  if (a.err[1] == 0) a.err[1] = 100 + site;
  *abort_flag = 1;
}

__global__ void __launch_bounds__(128, 1)
    chain_tc_kernel(const __grid_constant__ CUtensorMap tm_xh, const __grid_constant__ CUtensorMap tm_xl,
                    const __grid_constant__ CUtensorMap tm_ph, const __grid_constant__ CUtensorMap tm_pl,
                    const __grid_constant__ CUtensorMap tm_pth, const __grid_constant__ CUtensorMap tm_ptl,
                    const __grid_constant__ CUtensorMap tm_th, const __grid_constant__ CUtensorMap tm_tl,
                    const ChainArgs args) {
  const int BN = args.BN, m = args.m;
  const int nkc = m / CKC;
  const int nchunks = 2 * nkc;                  // term 1, then term 2
  const uint32_t b_bytes = (uint32_t)BN * 64;
  const uint32_t stage_bytes = 2 * CA_BYTES + 2 * b_bytes;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)CSTAGES * stage_bytes);
  uint64_t* empty = full + CSTAGES;
  uint64_t* done = empty + CSTAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * CBM, j0 = blockIdx.y * BN, s = blockIdx.z;
  const unsigned long long limit = args.timeout_ns;
  if (threadIdx.x == 0) {
    for (int q = 0; q < CSTAGES; ++q) {
      ptx::mbar_init(&full[q], 1);
      ptx::mbar_init(&empty[q], 1);
    }
    ptx::mbar_init(done, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, (uint32_t)BN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int prow = (s * args.kmax1 + args.k) * m;   // row of P_k / P_k^T in the power planes
  const int xrow = s * m;                            // row of X / X^T in the split planes

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    int armed[CSTAGES];
    for (int q = 0; q < CSTAGES; ++q) armed[q] = -1;
    for (int c = 0; c < nchunks && !*abort_flag; ++c) {
      const int q = c % CSTAGES;
      const uint32_t ph = (uint32_t)((c / CSTAGES) & 1);
      if (!ptx::mbar_wait(&empty[q], ph ^ 1u, limit, abort_flag)) {
        chain_fail(args, abort_flag, 1);
        break;
      }
      uint8_t* sa = smem + (size_t)q * stage_bytes;
      const int kx = (c % nkc) * CKC;
      ptx::mbar_arrive_expect_tx(&full[q], stage_bytes);
      if (c < nkc) {   // X P_k^T
        ptx::tma_load_2d(sa, &tm_xh, &full[q], kx, xrow + i0);
        ptx::tma_load_2d(sa + CA_BYTES, &tm_xl, &full[q], kx, xrow + i0);
        ptx::tma_load_2d(sa + 2 * CA_BYTES, &tm_ph, &full[q], kx, prow + j0);
        ptx::tma_load_2d(sa + 2 * CA_BYTES + b_bytes, &tm_pl, &full[q], kx, prow + j0);
      } else {         // P_k^T X
        ptx::tma_load_2d(sa, &tm_pth, &full[q], kx, prow + i0);
        ptx::tma_load_2d(sa + CA_BYTES, &tm_ptl, &full[q], kx, prow + i0);
        ptx::tma_load_2d(sa + 2 * CA_BYTES, &tm_th, &full[q], kx, xrow + j0);
        ptx::tma_load_2d(sa + 2 * CA_BYTES + b_bytes, &tm_tl, &full[q], kx, xrow + j0);
      }
      armed[q] = (int)ph;
    }
    // never leave with copies in flight
    for (int q = 0; q < CSTAGES; ++q)
      if (armed[q] >= 0) ptx::mbar_wait(&full[q], (uint32_t)armed[q], limit, nullptr);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = ptx::make_idesc(1u, CBM, BN);
    for (int c = 0; c < nchunks; ++c) {
      const int q = c % CSTAGES;
      const uint32_t ph = (uint32_t)((c / CSTAGES) & 1);
      if (!ptx::mbar_wait(&full[q], ph, limit, abort_flag)) {
        chain_fail(args, abort_flag, 2);
        break;
      }
      ptx::tc_fence_after();
      uint8_t* sa = smem + (size_t)q * stage_bytes;
      const uint64_t dah = ptx::make_sdesc_sw64(ptx::smem_addr(sa));
      const uint64_t dal = ptx::make_sdesc_sw64(ptx::smem_addr(sa + CA_BYTES));
      const uint64_t dbh = ptx::make_sdesc_sw64(ptx::smem_addr(sa + 2 * CA_BYTES));
      const uint64_t dbl = ptx::make_sdesc_sw64(ptx::smem_addr(sa + 2 * CA_BYTES + b_bytes));
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint64_t adv = (uint64_t)((kk * 32) >> 4);   // 16 BF16 = 32 bytes per MMA
        ptx::mma_bf16(tmem, dah + adv, dbh + adv, idesc, (c | kk) != 0);
        ptx::mma_bf16(tmem, dah + adv, dbl + adv, idesc, 1u);
        ptx::mma_bf16(tmem, dal + adv, dbh + adv, idesc, 1u);
      }
      ptx::tc_commit(&empty[q]);
    }
    ptx::tc_commit(done);   // every MMA issued above has completed when this arrives
  }
  __syncwarp();
  // ------------------------------------------------------------ epilogue (all warps)
  const bool ok = ptx::mbar_wait(done, 0u, 4 * limit, nullptr);
  ptx::tc_fence_after();
  // warp-uniform decision: the TMEM loads below are warp-collective
  if (__all_sync(0xffffffffu, ok && !*abort_flag)) {
    const int r = warp * 32 + lane;                  // tile row == TMEM lane
    const int i = i0 + r;
    float* out = args.dP + (int64_t)s * args.kst + (int64_t)args.k * m * m + (int64_t)i * m + j0;
    const int64_t xb = (int64_t)s * m * m;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      ptx::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      float4* o = reinterpret_cast<float4*>(out + c0);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float4 t = o[e];
        t.x += v[4 * e]; t.y += v[4 * e + 1]; t.z += v[4 * e + 2]; t.w += v[4 * e + 3];
        o[e] = t;
        v[4 * e] = t.x; v[4 * e + 1] = t.y; v[4 * e + 2] = t.z; v[4 * e + 3] = t.w;
      }
      if (args.oxh) {
        // dP_k is final here: its split planes feed the next level, as X (row i)
        // and as X^T (column i: the warp's 32 rows are 64 contiguous bytes per j)
        __nv_bfloat16 hv[32], lv[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          hv[e] = __float2bfloat16_rn(v[e]);
          lv[e] = __float2bfloat16_rn(v[e] - __bfloat162float(hv[e]));
        }
        uint4* xh4 = reinterpret_cast<uint4*>(args.oxh + xb + (int64_t)i * m + j0 + c0);
        uint4* xl4 = reinterpret_cast<uint4*>(args.oxl + xb + (int64_t)i * m + j0 + c0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          xh4[e] = *reinterpret_cast<const uint4*>(&hv[8 * e]);
          xl4[e] = *reinterpret_cast<const uint4*>(&lv[8 * e]);
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int64_t tix = xb + (int64_t)(j0 + c0 + e) * m + i;
          args.oth[tix] = hv[e];
          args.otl[tix] = lv[e];
        }
      }
    }
  } else if (!ok) {
    chain_fail(args, abort_flag, 3);
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem, (uint32_t)BN);
}

}  // namespace

bool chain_tc_supported(const Plan& p) {
  return p.d.precision == CASCADE_BF16_SPLIT && p.d.m % CBM == 0 && p.Phi && p.PThi;
}

size_t chain_tc_scratch_bytes(const Plan& p) {
  return (size_t)8 * p.d.nsys * p.d.m * p.d.m * sizeof(__nv_bfloat16);
}

// dP_k += dP_(k+1) P_k^T + P_k^T dP_(k+1) for every system.  scratch holds two sets
// of the four split planes (chain_tc_scratch_bytes): level k reads set k & 1 (split
// here from dP_(k+1) on the first level, first = true) and its epilogue writes the
// planes of the finished dP_k into the other set for level k - 1.
cudaError_t launch_chain_tc(const Plan& p, int k, bool first, float* dP, int64_t kst,
                            void* scratch, cudaStream_t st) {
  const int m = p.d.m, ns = p.d.nsys;
  const int64_t mm = (int64_t)m * m;
  __nv_bfloat16* set0 = static_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* xh = set0 + (int64_t)(k & 1) * 4 * ns * mm;
  __nv_bfloat16* xl = xh + ns * mm;
  __nv_bfloat16* th = xl + ns * mm;
  __nv_bfloat16* tl = th + ns * mm;
  __nv_bfloat16* oh = set0 + (int64_t)((k + 1) & 1) * 4 * ns * mm;
  if (first) {
    chain_split_kernel<<<dim3(m / 32, m / 32, ns), dim3(32, 8), 0, st>>>(
        dP + (int64_t)(k + 1) * mm, kst, m, xh, xl, th, tl);
    CASCADE_LAUNCHED();
  }
  // column blocks narrow enough to occupy every SM, down to 64 (narrower
  // blocks would read more operand bytes per product than shared memory
  // delivers): one level is a small product (12 m^3 flops per system), which
  // blocks of 256 columns spread over 32 SMs at m = 1024 and over 2 at m = 256
  int BN = 256;
  while (BN > 64 && (m % BN != 0 || (int64_t)(m / CBM) * (m / BN) * ns < p.num_sms)) BN /= 2;
  CUtensorMap maps[8];
  std::string err;
  const uint64_t xrows = (uint64_t)ns * m, prows = (uint64_t)ns * p.kmax1 * m;
  if (!encode_tmap_2d(&maps[0], xh, 2, m, xrows, CKC, CBM, &err, 64) ||
      !encode_tmap_2d(&maps[1], xl, 2, m, xrows, CKC, CBM, &err, 64) ||
      !encode_tmap_2d(&maps[2], p.Phi, 2, m, prows, CKC, BN, &err, 64) ||
      !encode_tmap_2d(&maps[3], p.Plo, 2, m, prows, CKC, BN, &err, 64) ||
      !encode_tmap_2d(&maps[4], p.PThi, 2, m, prows, CKC, CBM, &err, 64) ||
      !encode_tmap_2d(&maps[5], p.PTlo, 2, m, prows, CKC, CBM, &err, 64) ||
      !encode_tmap_2d(&maps[6], th, 2, m, xrows, CKC, BN, &err, 64) ||
      !encode_tmap_2d(&maps[7], tl, 2, m, xrows, CKC, BN, &err, 64)) {
    set_global_error("tensor map encode failed: " + err);
    return cudaErrorInvalidValue;
  }
  ChainArgs a{};
  a.m = m;
  a.kmax1 = p.kmax1;
  a.k = k;
  a.BN = BN;
  a.dP = dP;
  a.kst = kst;
  if (k > 0) {   // dP_0 feeds no further level
    a.oxh = oh;
    a.oxl = oh + ns * mm;
    a.oth = oh + 2 * ns * mm;
    a.otl = oh + 3 * ns * mm;
  }
  a.err = p.err;
  a.timeout_ns = 2000000000ull;
  const size_t smem = 1024 + (size_t)CSTAGES * (2 * CA_BYTES + 2 * (size_t)BN * 64) +
                      8 * (2 * CSTAGES + 1) + 16;
  cudaError_t e = cudaFuncSetAttribute(chain_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  chain_tc_kernel<<<dim3(m / CBM, m / BN, ns), 128, smem, st>>>(
      maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6], maps[7], a);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace cascade
