// stage_simt.cu -- cascade kernels on the CUDA cores:
//   * the first stage fused with the input projection,
//       v^(1)_l = Bbar u_l + (Abar Bbar) u_(l-1)      (§3: v^(0) = Bbar u, Eq. 3.2),
//     so v^(0) never exists in memory and the m x m product of stage 0 becomes
//     an m x 2p one;
//   * the FP64 stage v_l <- v_l + P v_(l-s) (general step of §3) for the FP64
//     path, tiled 64 x 64 with FP64 FMAs;
//   * the output projection y = C v + D u (end of §3) where it is not fused;
//   * the FP64 sequential recursion of Eq. (1.2), the baseline the cascade
//     replaces;
//   * a bounded-wait self-test.
#include "common.cuh"
#include "formats.cuh"
#include "ptx.cuh"

namespace cascade {
namespace {

// ---------------------------------------------------------------- first stage
// One block per tile of BM rows; thread items (row, column) with the column
// fastest.  T is the element type of u and of the coefficient matrices.
template <int FMT, typename T>
__global__ void __launch_bounds__(256) stage0_kernel(const Tile* __restrict__ tiles, int BM, int m,
                                                     int p, const T* __restrict__ u,
                                                     const T* __restrict__ Bbar,
                                                     const T* __restrict__ ABbar, void* out_hi,
                                                     void* out_lo) {
  const Tile t = tiles[blockIdx.x];
  const int rows = min(BM, t.len - t.t0);
  const T* Bs = Bbar + (int64_t)t.sys * m * p;
  const T* ABs = ABbar + (int64_t)t.sys * m * p;
  for (int64_t idx = threadIdx.x; idx < (int64_t)rows * m; idx += blockDim.x) {
    const int r = (int)(idx / m), c = (int)(idx % m);
    const int l = t.t0 + r;
    const int64_t row = t.seq_row0 + l;
    const T* ur = u + row * p;
    double acc = 0.0;
    for (int j = 0; j < p; ++j) acc = fma((double)Bs[(int64_t)c * p + j], (double)ur[j], acc);
    if (l >= 1) {
      const T* up = ur - p;
      for (int j = 0; j < p; ++j) acc = fma((double)ABs[(int64_t)c * p + j], (double)up[j], acc);
    }
    Store<FMT>::put(out_hi, out_lo, row * m + c, acc);
  }
}

// First stage for the tensor-core formats: one thread writes 8 consecutive
// state entries of one row (16-byte stores per plane), FP32 arithmetic.
// Requires m % 8 == 0 (the tensor-core precisions need m % 32 == 0).
template <int FMT>
__global__ void __launch_bounds__(256) stage0_vec_kernel(const Tile* __restrict__ tiles, int BM,
                                                         int m, int p, const float* __restrict__ u,
                                                         const float* __restrict__ Bbar,
                                                         const float* __restrict__ ABbar,
                                                         void* out_hi, void* out_lo) {
  const Tile t = tiles[blockIdx.x];
  const int rows = min(BM, t.len - t.t0);
  const int groups = m >> 3;
  const float* Bs = Bbar + (int64_t)t.sys * m * p;
  const float* ABs = ABbar + (int64_t)t.sys * m * p;
  for (int idx = threadIdx.x; idx < rows * groups; idx += blockDim.x) {
    const int r = idx / groups, c0 = (idx % groups) * 8;
    const int l = t.t0 + r;
    const int64_t row = t.seq_row0 + l;
    const float* ur = u + row * p;
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
    for (int j = 0; j < p; ++j) {
      const float uj = __ldg(ur + j);
      const float upj = l >= 1 ? __ldg(ur - p + j) : 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        acc[e] = fmaf(__ldg(Bs + (int64_t)(c0 + e) * p + j), uj,
                      fmaf(__ldg(ABs + (int64_t)(c0 + e) * p + j), upj, acc[e]));
    }
    const int64_t off = row * m + c0;
    if (FMT == FMT_BF16) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(acc[2 * j], acc[2 * j + 1]);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(acc[2 * j] - hf.x, acc[2 * j + 1] - hf.y);
        hw[j] = *reinterpret_cast<const uint32_t*>(&hh);
        lw[j] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out_hi) + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out_lo) + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    } else {
      float hv[8], lv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        hv[e] = ptx::tf32_rna(acc[e]);
        lv[e] = ptx::tf32_rna(acc[e] - hv[e]);
      }
      float4* h = reinterpret_cast<float4*>(static_cast<float*>(out_hi) + off);
      float4* lo4 = reinterpret_cast<float4*>(static_cast<float*>(out_lo) + off);
      h[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
      h[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
      lo4[0] = make_float4(lv[0], lv[1], lv[2], lv[3]);
      lo4[1] = make_float4(lv[4], lv[5], lv[6], lv[7]);
    }
  }
}

// ---------------------------------------------------------------- FP64 stage
// Block: 64 rows x NB state columns of one tile, 256 threads, 4 x (NB / 16) outputs
// each.  NB = 64, or 32 / 16 when a stage has too few tiles to fill the GPU.
template <int NB>
__global__ void __launch_bounds__(256) stage_f64_kernel(const Tile* __restrict__ tiles, int m,
                                                        int shift, int reverse,
                                                        const double* __restrict__ P,
                                                        int64_t p_sys_stride,
                                                        const double* __restrict__ vin,
                                                        double* __restrict__ vout) {
  constexpr int BMF = 64;
  constexpr int NJ = NB / 16;
  __shared__ double As[16][65];   // [k][row]
  __shared__ double Bs[16][NB + 1];   // [k][col]
  const Tile t = tiles[blockIdx.x];
  const int n0 = blockIdx.y * NB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double* Ps = P + (int64_t)t.sys * p_sys_stride;
  // adjoint stages (reverse): source l + s and the transposed power
  const bool copy = reverse ? (t.t0 + shift >= t.len) : (t.t0 + BMF <= shift);
  double acc[4][NJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0;
  if (!copy) {
    for (int k0 = 0; k0 < m; k0 += 16) {
      for (int e = threadIdx.x; e < 1024; e += 256) {
        const int kk = e & 15, rr = e >> 4;
        const int l = t.t0 + rr + (reverse ? shift : -shift);   // source time step
        const int gk = k0 + kk;
        double v = 0.0;
        if (l >= 0 && l < t.len && t.t0 + rr < t.len && gk < m)
          v = vin[(t.seq_row0 + l) * (int64_t)m + gk];
        As[kk][rr] = v;
      }
      for (int e = threadIdx.x; e < 16 * NB; e += 256) {
        const int kk = e & 15, nn = e >> 4;
        const int gn = n0 + nn, gk = k0 + kk;
        Bs[kk][nn] = (gn < m && gk < m) ? Ps[(int64_t)gn * m + gk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        double a[4], b[NJ];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < NJ; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = ty + 16 * i;
    if (t.t0 + rr >= t.len) continue;
    const int64_t row = t.seq_row0 + t.t0 + rr;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= m) continue;
      vout[row * m + gn] = vin[row * m + gn] + acc[i][j];
    }
  }
}

// ---------------------------------------------------------------- output
// One block per output tile (tile.fbuf = which workspace buffer holds the
// final states); one warp per row: y[row, :] = C v + D u.
template <int FMT, typename T>
__global__ void __launch_bounds__(256) output_kernel(const Tile* __restrict__ tiles, int BM, int m,
                                                     int p, int q, const T* __restrict__ u,
                                                     T* __restrict__ y, const T* __restrict__ C,
                                                     const T* __restrict__ D, Bufs V) {
  const Tile t = tiles[blockIdx.x];
  const void* vh = V.hi(t.fbuf);
  const void* vl = V.lo(t.fbuf);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int rows = min(BM, t.len - t.t0);
  const T* Cs = C + (int64_t)t.sys * q * m;
  const T* Ds = D + (int64_t)t.sys * q * p;
  for (int r = warp; r < rows; r += nw) {
    const int64_t row = t.seq_row0 + t.t0 + r;
    for (int q0 = 0; q0 < q; q0 += 8) {
      T acc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] = 0;
      for (int c = lane; c < m; c += 32) {
        const T v = (T)load_elem<FMT>(vh, vl, row * m + c);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (q0 + i < q) acc[i] = fma(Cs[(int64_t)(q0 + i) * m + c], v, acc[i]);
      }
      for (int c = lane; c < p; c += 32) {
        const T uv = u[row * p + c];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (q0 + i < q) acc[i] = fma(Ds[(int64_t)(q0 + i) * p + c], uv, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        T s = acc[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0 && q0 + i < q) y[row * q + q0 + i] = (T)s;
      }
    }
  }
}

// ---------------------------------------------------------------- recursion
// Eq. (1.2) one step at a time: x_n = Abar x_(n-1) + Bbar u_n, y_n = C x_n + D u_n.
// One block per sequence; the state lives in shared memory (double buffer).
__global__ void __launch_bounds__(256) recursion_f64_kernel(const Seq* __restrict__ seqs, int m,
                                                            int p, int q,
                                                            const double* __restrict__ Abar,
                                                            int64_t a_sys_stride,
                                                            const double* __restrict__ Bbar,
                                                            const double* __restrict__ C,
                                                            const double* __restrict__ D,
                                                            const double* __restrict__ u,
                                                            double* __restrict__ y) {
  extern __shared__ double xs[];   // 2 * m
  const Seq sq = seqs[blockIdx.x];
  const double* As = Abar + (int64_t)sq.sys * a_sys_stride;
  const double* Bs = Bbar + (int64_t)sq.sys * m * p;
  const double* Cs = C + (int64_t)sq.sys * q * m;
  const double* Ds = D + (int64_t)sq.sys * q * p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* x = xs;
  double* xn = xs + m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] = 0.0;
  __syncthreads();
  for (int l = 0; l < sq.len; ++l) {
    const double* ur = u + (sq.row0 + l) * p;
    for (int i = warp; i < m; i += nw) {
      double s = 0.0;
      for (int j = lane; j < m; j += 32) s = fma(As[(int64_t)i * m + j], x[j], s);
      for (int j = lane; j < p; j += 32) s = fma(Bs[(int64_t)i * p + j], ur[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) xn[i] = s;
    }
    __syncthreads();
    for (int qq = warp; qq < q; qq += nw) {
      double s = 0.0;
      for (int j = lane; j < m; j += 32) s = fma(Cs[(int64_t)qq * m + j], xn[j], s);
      for (int j = lane; j < p; j += 32) s = fma(Ds[(int64_t)qq * p + j], ur[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) y[(sq.row0 + l) * q + qq] = s;
    }
    double* tmp = x;
    x = xn;
    xn = tmp;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- self-test
// Waits on an mbarrier that nothing arrives at; the bounded wait must give up.
__global__ void selftest_timeout_kernel(unsigned long long limit_ns, int32_t* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = ptx::mbar_wait(&bar, 0u, limit_ns, &abort_flag);
    *err = ok ? 0 : (int32_t)CASCADE_ERR_TIMEOUT;
  }
}

}  // namespace

cudaError_t launch_stage0(const Plan& p, const void* u, void* out_hi, void* out_lo,
                          cudaStream_t st) {
  const int n = p.n_stage0_tiles;
  if (n == 0) return cudaSuccess;
  const int BM = tile_rows(p);
  switch (p.d.precision) {
    case CASCADE_FP64:
      stage0_kernel<FMT_F64, double><<<n, 256, 0, st>>>(p.d_stage0_tiles, BM, p.d.m, p.d.p,
                                                        (const double*)u, p.Bbar64, p.ABbar64,
                                                        out_hi, out_lo);
      break;
    case CASCADE_BF16_SPLIT:
      stage0_vec_kernel<FMT_BF16><<<n, 256, 0, st>>>(p.d_stage0_tiles, BM, p.d.m, p.d.p,
                                                     (const float*)u, p.Bbar32, p.ABbar32,
                                                     out_hi, out_lo);
      break;
    default:
      stage0_vec_kernel<FMT_F32><<<n, 256, 0, st>>>(p.d_stage0_tiles, BM, p.d.m, p.d.p,
                                                    (const float*)u, p.Bbar32, p.ABbar32,
                                                    out_hi, out_lo);
  }
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_stage_f64(const Plan& p, int k, const double* vin, double* vout,
                             cudaStream_t st, bool reverse) {
  const int n = reverse ? p.n_adj_tiles[k] : p.n_tiles[k];
  if (n == 0) return cudaSuccess;
  if (!(reverse ? p.PT64 : p.P64) || !vin || !vout) {
    set_global_error("stage launch without its powers or state buffers");
    return cudaErrorInvalidValue;
  }
  // column blocks of 64, or narrower while a launch would leave SMs idle
  int nb = 64;
  while (nb > 16 && (int64_t)n * ((p.d.m + nb - 1) / nb) < p.num_sms) nb >>= 1;
  const Tile* tl = reverse ? p.d_adj_tiles[k] : p.d_tiles[k];
  const double* Pk = (reverse ? p.PT64 : p.P64) + (int64_t)k * p.d.m * p.d.m;
  const int64_t pss = (int64_t)p.kmax1 * p.d.m * p.d.m;
  const dim3 grid(n, (p.d.m + nb - 1) / nb);
  if (nb == 64)
    stage_f64_kernel<64><<<grid, 256, 0, st>>>(tl, p.d.m, 1 << k, reverse ? 1 : 0, Pk, pss, vin, vout);
  else if (nb == 32)
    stage_f64_kernel<32><<<grid, 256, 0, st>>>(tl, p.d.m, 1 << k, reverse ? 1 : 0, Pk, pss, vin, vout);
  else
    stage_f64_kernel<16><<<grid, 256, 0, st>>>(tl, p.d.m, 1 << k, reverse ? 1 : 0, Pk, pss, vin, vout);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_output(const Plan& p, const void* u, void* y, const Bufs& V, cudaStream_t st) {
  const int n = p.n_out_tiles;
  if (n == 0) return cudaSuccess;
  const int BM = tile_rows(p);
  const Tile* tiles = p.d_out_tiles;
  switch (p.d.precision) {
    case CASCADE_FP64:
      output_kernel<FMT_F64, double><<<n, 256, 0, st>>>(tiles, BM, p.d.m, p.d.p, p.d.q,
                                                        (const double*)u, (double*)y, p.C64,
                                                        p.D64, V);
      break;
    case CASCADE_BF16_SPLIT:
      output_kernel<FMT_BF16, float><<<n, 256, 0, st>>>(tiles, BM, p.d.m, p.d.p, p.d.q,
                                                        (const float*)u, (float*)y, p.C32, p.D32,
                                                        V);
      break;
    default:
      output_kernel<FMT_F32, float><<<n, 256, 0, st>>>(tiles, BM, p.d.m, p.d.p, p.d.q,
                                                       (const float*)u, (float*)y, p.C32, p.D32,
                                                       V);
  }
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_recursion_f64(const Plan& p, const double* u, double* y, cudaStream_t st) {
  if (p.nseq == 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(double) * (size_t)p.d.m;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(recursion_f64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  recursion_f64_kernel<<<p.nseq, 256, smem, st>>>(p.d_seqs, p.d.m, p.d.p, p.d.q, p.P64,
                                                  (int64_t)p.kmax1 * p.d.m * p.d.m, p.Bbar64,
                                                  p.C64, p.D64, u, y);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_selftest_timeout(int32_t limit_us, int32_t* err, cudaStream_t st) {
  selftest_timeout_kernel<<<1, 32, 0, st>>>((unsigned long long)limit_us * 1000ull, err);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace cascade
