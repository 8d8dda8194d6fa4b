// precompute.cu -- FP64 system preparation on the device:
//   trapezoidal discretisation (§1 after Eq. 1.2, Eq. 4.2),
//   powers Abar^(2^k) by repeated squaring (end of §2, §4),
//   Frobenius norms for the accuracy rule (Lemma 1, remainder reading),
//   conversion of the powers into tensor-core operand planes (hi + lo).
#include "common.cuh"

#include <math.h>

#include <algorithm>

namespace cascade {

// ----------------------------------------------------------------------------
// Discretisation: one thread block per system solves
//   (I - delta/2 A) [Abar | Bbar | M^-1] = [I + delta/2 A | delta B | I]
// by Gauss-Jordan elimination with partial pivoting, in FP64, on an augmented
// m x (3m + p) matrix held in global memory (M^-1 feeds the adjoint).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) discretise_kernel(
    const double* __restrict__ A, const double* __restrict__ B, const double* __restrict__ delta,
    const double* __restrict__ scale, double* __restrict__ Abar, int64_t abar_stride,
    double* __restrict__ Bbar, double* __restrict__ Minv, double* __restrict__ work, int m, int p,
    int32_t* singular, int lower) {
  extern __shared__ double fac[];          // m elimination factors
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv;
  __shared__ double s_inv;
  const int s = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int W = 3 * m + p;
  const double dl = delta[s];
  const double h = 0.5 * dl;
  const double* As = A + (int64_t)s * m * m;
  const double* Bs = B + (int64_t)s * m * p;
  double* T = work + (int64_t)s * m * W;

  for (int64_t idx = tid; idx < (int64_t)m * W; idx += nt) {
    const int i = (int)(idx / W), j = (int)(idx % W);
    double v;
    if (j < m) v = (i == j ? 1.0 : 0.0) - h * As[(int64_t)i * m + j];
    else if (j < 2 * m) v = (i == j - m ? 1.0 : 0.0) + h * As[(int64_t)i * m + (j - m)];
    else if (j < 2 * m + p) v = dl * Bs[(int64_t)i * p + (j - 2 * m)];
    else v = (i == j - 2 * m - p) ? 1.0 : 0.0;
    T[idx] = v;
  }
  __syncthreads();

  // lower (A lower-triangular, so M = I - delta/2 A is): a triangular system
  // needs no row exchanges (forward elimination without them is backward
  // stable), so the pivot is the diagonal.  In the three triangular blocks (M,
  // I + delta/2 A, I) row c is then zero past offset c and the rows above c have
  // a zero in column c, so the elimination touches rows below c and, in those
  // blocks, offsets up to c only; the result is exactly lower-triangular.  When
  // the dense elimination exchanges no rows either, the two agree bit for bit.
  for (int c = 0; c < m; ++c) {
    if (lower) {
      if (tid == 0) {
        s_piv = c;
        if (!(T[(int64_t)c * W + c] != 0.0)) atomicExch(singular, 1);
      }
    } else {
      // pivot: largest |T[i][c]| for i >= c (smallest index on ties)
      double best = -1.0;
      int bi = c;
      for (int i = c + tid; i < m; i += nt) {
        const double a = fabs(T[(int64_t)i * W + c]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
      __syncthreads();
      if (tid == 0) {
        double b = red_v[0];
        int i0 = red_i[0];
        for (int w = 1; w < (nt + 31) / 32; ++w)
          if (red_v[w] > b || (red_v[w] == b && red_i[w] < i0)) { b = red_v[w]; i0 = red_i[w]; }
        s_piv = i0;
        if (!(b > 0.0)) atomicExch(singular, 1);
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != c) {
      for (int j = c + tid; j < W; j += nt) {
        const double t = T[(int64_t)c * W + j];
        T[(int64_t)c * W + j] = T[(int64_t)piv * W + j];
        T[(int64_t)piv * W + j] = t;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double d = T[(int64_t)c * W + c];
      s_inv = d != 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    // columns of row c that may be non-zero: all W - c of them, or with lower
    // column c of M, offsets 0..c of the other two triangular blocks and all of B
    const int nc = lower ? 1 + (c + 1) + p + (c + 1) : W - c;
    auto col = [&](int t) -> int {
      if (!lower) return c + t;
      if (t == 0) return c;
      t -= 1;
      if (t <= c) return m + t;
      t -= c + 1;
      if (t < p) return 2 * m + t;
      return 2 * m + p + (t - p);
    };
    for (int t = tid; t < nc; t += nt) T[(int64_t)c * W + col(t)] *= inv;
    for (int i = tid; i < m; i += nt) fac[i] = (i == c) ? 0.0 : T[(int64_t)i * W + c];
    __syncthreads();
    const int r0 = lower ? c + 1 : 0;                 // rows that may hold a non-zero factor
    const int64_t nupd = (int64_t)(m - r0) * nc;
    for (int64_t idx = tid; idx < nupd; idx += nt) {
      const int i = r0 + (int)(idx / nc), j = col((int)(idx % nc));
      const double f = fac[i];
      if (f != 0.0) T[(int64_t)i * W + j] -= f * T[(int64_t)c * W + j];
    }
    __syncthreads();
  }

  const double sc = scale ? scale[s] : 1.0;
  double* Ab = Abar + (int64_t)s * abar_stride;
  for (int64_t idx = tid; idx < (int64_t)m * m; idx += nt) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    Ab[idx] = sc * T[(int64_t)i * W + m + j];
  }
  double* Bb = Bbar + (int64_t)s * m * p;
  for (int64_t idx = tid; idx < (int64_t)m * p; idx += nt) {
    const int i = (int)(idx / p), j = (int)(idx % p);
    Bb[idx] = T[(int64_t)i * W + 2 * m + j];
  }
  if (Minv) {
    double* Mi = Minv + (int64_t)s * m * m;
    for (int64_t idx = tid; idx < (int64_t)m * m; idx += nt) {
      const int i = (int)(idx / m), j = (int)(idx % m);
      Mi[idx] = T[(int64_t)i * W + 2 * m + p + j];
    }
  }
}

cudaError_t launch_discretise(const double* A, const double* B, const double* delta,
                              const double* scale, double* Abar_out, int64_t abar_sys_stride,
                              double* Bbar_out, double* Minv_out, double* work, int nsys, int m,
                              int p, int32_t* singular, bool lower, cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)m;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(discretise_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  discretise_kernel<<<nsys, 1024, smem, st>>>(A, B, delta, scale, Abar_out, abar_sys_stride,
                                               Bbar_out, Minv_out, work, m, p, singular,
                                               lower ? 1 : 0);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Batched FP64 GEMM  C = alpha op(A) op(B) + beta C  (row-major), TM x TM tiles
// (64, or 32 when 64-wide tiles would leave the grid short of a few waves),
// (TM / 16)^2 outputs per thread.  Used for the squaring chain P_{k+1} = P_k P_k,
// the product Abar Bbar, and the adjoint of the squaring chain.
// ----------------------------------------------------------------------------
template <typename T, bool TA, bool TB, int TM = 64>
__global__ void __launch_bounds__(256) gemm_kernel(const T* __restrict__ A, const T* __restrict__ B,
                                                   T* __restrict__ C, int M, int N, int K, int lda,
                                                   int ldb, int ldc, int64_t sA, int64_t sB,
                                                   int64_t sC, T alpha, T beta, int lower = 0) {
  constexpr int R = TM / 16;       // outputs per thread along each axis
  __shared__ T As[16][TM + 1];
  __shared__ T Bs[16][TM + 1];
  A += (int64_t)blockIdx.z * sA;
  B += (int64_t)blockIdx.z * sB;
  C += (int64_t)blockIdx.z * sC;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0;

  // lower: A and B lower-triangular (C = A B is too).  A tile above the diagonal
  // is zero, and the K loop runs over k in [n0, m0 + 64) only: every product left
  // out has an exactly zero factor, so the sums are the full loop's bit for bit.
  int kbeg = 0, kend = K;
  if (lower) {
    kbeg = n0 < m0 + TM ? n0 : 0;
    kend = n0 < m0 + TM ? min(K, m0 + TM) : 0;
  }
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * TM; e += 256) {
      int mm, kk;
      if (!TA) { kk = e & 15; mm = e >> 4; } else { mm = e % TM; kk = e / TM; }
      const int gm = m0 + mm, gk = k0 + kk;
      T v = 0;
      if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < 16 * TM; e += 256) {
      int nn, kk;
      if (!TB) { nn = e % TM; kk = e / TM; } else { kk = e & 15; nn = e >> 4; }
      const int gn = n0 + nn, gk = k0 + kk;
      T v = 0;
      if (gn < N && gk < K) v = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      T* c = C + (int64_t)gm * ldc + gn;
      *c = alpha * acc[i][j] + (beta != (T)0 ? beta * *c : (T)0);
    }
  }
}

template <typename T>
cudaError_t launch_gemm(const T* A, const T* B, T* C, int M, int N, int K, int lda, int ldb,
                        int ldc, int64_t sA, int64_t sB, int64_t sC, int batch, T alpha, T beta,
                        bool transA, bool transB, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  // 32-wide tiles when 64-wide ones would give fewer than four blocks per SM
  // (one system of m = 1024: 256 blocks on 152 SMs, a second wave two thirds full)
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 1;
  }
  const int64_t blocks64 = (int64_t)((N + 63) / 64) * ((M + 63) / 64) * batch;
  if (blocks64 < 4 * (int64_t)nsm) {
    dim3 grid((N + 31) / 32, (M + 31) / 32, batch);
    if (!transA && !transB)
      gemm_kernel<T, false, false, 32><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
    else if (transA && !transB)
      gemm_kernel<T, true, false, 32><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
    else if (!transA && transB)
      gemm_kernel<T, false, true, 32><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
    else
      gemm_kernel<T, true, true, 32><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
    CASCADE_LAUNCHED();
    return cudaGetLastError();
  }
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  if (!transA && !transB)
    gemm_kernel<T, false, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
  else if (transA && !transB)
    gemm_kernel<T, true, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
  else if (!transA && transB)
    gemm_kernel<T, false, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
  else
    gemm_kernel<T, true, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, alpha, beta);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

// flag = 1 if any of the ns matrices X[s] (m x m, row-major, sys_stride apart)
// has a non-zero entry above the diagonal (flag is not cleared here).
__global__ void upper_nonzero_kernel(const double* __restrict__ X, int64_t sys_stride, int ns,
                                     int m, int32_t* flag) {
  const int64_t mm = (int64_t)m * m, n = mm * ns;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / mm, r = idx % mm;
    if (r % m > r / m && X[s * sys_stride + r] != 0.0) *flag = 1;
  }
}

cudaError_t launch_upper_nonzero(const double* X, int64_t sys_stride, int ns, int m, int32_t* flag,
                                 cudaStream_t st) {
  if (ns <= 0 || m <= 0) return cudaSuccess;
  const int64_t n = (int64_t)ns * m * m;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  upper_nonzero_kernel<<<grid, 256, 0, st>>>(X, sys_stride, ns, m, flag);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_dgemm_lower(const double* A, const double* B, double* C, int n, int64_t sA,
                               int64_t sB, int64_t sC, int batch, cudaStream_t st) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  // 32-wide tiles: the products of the tiles that straddle the diagonal, half of
  // which have a zero factor, are 1.4x the triangle's (1.9x with 64-wide tiles)
  dim3 grid((n + 31) / 32, (n + 31) / 32, batch);
  gemm_kernel<double, false, false, 32><<<grid, 256, 0, st>>>(A, B, C, n, n, n, n, n, n, sA, sB,
                                                              sC, 1.0, 0.0, 1);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_dgemm(const double* A, const double* B, double* C, int M, int N, int K,
                         int lda, int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC,
                         int batch, double alpha, double beta, bool transA, bool transB,
                         cudaStream_t st) {
  return launch_gemm<double>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, alpha, beta,
                             transA, transB, st);
}

// ----------------------------------------------------------------------------
// Batched FP32 GEMM with two products, C = alpha (op(A1) op(B1) + op(A2) op(B2))
// + beta C (row-major; A2 may be null), 128 x 128 tiles, 8 x 8 outputs per
// thread as two 4 x 4 quadrants (float4 shared-memory reads).  Used for the
// backward's squaring-chain adjoint dP_k += dP_(k+1) P_k^T + P_k^T dP_(k+1),
// one launch per level.
// ----------------------------------------------------------------------------
struct GemmOp {
  const float* A;
  const float* B;
  int lda, ldb;
  int64_t sA, sB;
  int ta, tb;
};

constexpr int G2_BK = 16;

// dst[k][r] = op(X)[r0 + r][k0 + k] for r < TBM, k < 16; op(X)[r][k] = trans ? X[k][r] : X[r][k]
template <int TBM>
__device__ __forceinline__ void g2_load(float (*dst)[TBM + 4], const float* X, int ld, bool trans,
                                        int r0, int k0, int R, int Kend) {
  constexpr int PER = TBM * G2_BK / 256;   // elements per thread: 8 or 4
  const int t = threadIdx.x;
  if (!trans) {
    constexpr int TPR = G2_BK / PER;       // threads per row
    const int r = t / TPR, kb = (t % TPR) * PER;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int gr = r0 + r, gk = k0 + kb + e;
      dst[kb + e][r] = (gr < R && gk < Kend) ? X[(int64_t)gr * ld + gk] : 0.f;
    }
  } else {
    constexpr int TPK = TBM / PER;         // threads per k
    const int k = t / TPK, rb = (t % TPK) * PER;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int gr = r0 + rb + e, gk = k0 + k;
      dst[k][rb + e] = (gr < R && gk < Kend) ? X[(int64_t)gk * ld + gr] : 0.f;
    }
  }
}

// TBM = 128: 8 x 8 outputs per thread (two 4 x 4 quadrants); TBM = 64: 4 x 4.
// gridDim.z = batch * ks: slice z % ks of K; with ks > 1 the slice's product
// (times alpha) goes to part[slice][b] and a second kernel adds the slices in
// order (deterministic split-K).
template <int TBM>
__global__ void __launch_bounds__(256, 2) sgemm2_kernel(GemmOp o1, GemmOp o2, int two,
                                                     float* __restrict__ C, int M, int N, int K,
                                                     int ldc, int64_t sC, float alpha,
                                                     float beta, int ks,
                                                     float* __restrict__ part) {
  constexpr int Q = TBM / 32;   // outputs per thread per dimension / 2 quadrants (4 or 2)
  constexpr int T = TBM == 128 ? 8 : 4;
  __shared__ __align__(16) float As[G2_BK][TBM + 4];
  __shared__ __align__(16) float Bs[G2_BK][TBM + 4];
  const int b = blockIdx.z / ks, slice = blockIdx.z % ks;
  const int kc = ((K + ks - 1) / ks + G2_BK - 1) / G2_BK * G2_BK;
  const int kbeg = slice * kc, kend = min(K, kbeg + kc);
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[T][T];
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int j = 0; j < T; ++j) acc[i][j] = 0.f;
  // row (column) of output i: quadrant i / 4 at offset TBM / 2, then 4 consecutive
  auto rix = [&](int i, int tid) { return (i >> 2) * (TBM / 2) + tid * 4 + (i & 3); };
  for (int op = 0; op < 1 + two; ++op) {
    const GemmOp& o = op ? o2 : o1;
    const float* A = o.A + (int64_t)b * o.sA;
    const float* B = o.B + (int64_t)b * o.sB;
    for (int k0 = kbeg; k0 < kend; k0 += G2_BK) {
      g2_load<TBM>(As, A, o.lda, o.ta != 0, m0, k0, M, kend);
      // op(B)[k][n] = op(B^T)[n][k]: load B^T's rows n with the opposite transposition
      g2_load<TBM>(Bs, B, o.ldb, o.tb == 0, n0, k0, N, kend);
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < G2_BK; ++kk) {
        float a[T], bv[T];
#pragma unroll
        for (int h = 0; h < T / 4; ++h) {
          const float4 av = *reinterpret_cast<const float4*>(&As[kk][h * (TBM / 2) + ty * 4]);
          const float4 bw = *reinterpret_cast<const float4*>(&Bs[kk][h * (TBM / 2) + tx * 4]);
          a[4 * h] = av.x; a[4 * h + 1] = av.y; a[4 * h + 2] = av.z; a[4 * h + 3] = av.w;
          bv[4 * h] = bw.x; bv[4 * h + 1] = bw.y; bv[4 * h + 2] = bw.z; bv[4 * h + 3] = bw.w;
        }
#pragma unroll
        for (int i = 0; i < T; ++i)
#pragma unroll
          for (int j = 0; j < T; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  (void)Q;
  if (ks == 1) {
    float* Cb = C + (int64_t)b * sC;
#pragma unroll
    for (int i = 0; i < T; ++i) {
      const int gm = m0 + rix(i, ty);
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        const int gn = n0 + rix(j, tx);
        if (gn >= N) continue;
        float* cp = Cb + (int64_t)gm * ldc + gn;
        *cp = alpha * acc[i][j] + (beta != 0.f ? beta * *cp : 0.f);
      }
    }
  } else {
    const int batch = gridDim.z / ks;
    float* Pb = part + ((int64_t)slice * batch + b) * M * N;
#pragma unroll
    for (int i = 0; i < T; ++i) {
      const int gm = m0 + rix(i, ty);
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        const int gn = n0 + rix(j, tx);
        if (gn < N) Pb[(int64_t)gm * N + gn] = alpha * acc[i][j];
      }
    }
  }
}

// C[b] = beta C[b] + sum over slices, in order, of part[slice][b]
__global__ void splitk_sum_kernel(const float* __restrict__ part, int ks, int batch, int M, int N,
                                  float* __restrict__ C, int ldc, int64_t sC, float beta) {
  const int b = blockIdx.y;
  const int64_t mn = (int64_t)M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mn;
       e += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int sl = 0; sl < ks; ++sl) v += part[((int64_t)sl * batch + b) * mn + e];
    float* cp = C + (int64_t)b * sC + (e / N) * ldc + (e % N);
    *cp = (beta != 0.f ? beta * *cp : 0.f) + v;
  }
}

cudaError_t launch_sgemm2(const float* A1, const float* B1, bool tA1, bool tB1, const float* A2,
                          const float* B2, bool tA2, bool tB2, float* C, int M, int N, int K,
                          int lda, int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC,
                          int batch, float alpha, float beta, cudaStream_t st, float* scratch,
                          size_t scratch_floats) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  const GemmOp o1{A1, B1, lda, ldb, sA, sB, tA1 ? 1 : 0, tB1 ? 1 : 0};
  const GemmOp o2{A2 ? A2 : A1, B2 ? B2 : B1, lda, ldb, sA, sB, tA2 ? 1 : 0, tB2 ? 1 : 0};
  const int64_t tiles128 = (int64_t)((M + 127) / 128) * ((N + 127) / 128) * batch;
  if (tiles128 >= sms) {
    dim3 grid((N + 127) / 128, (M + 127) / 128, batch);
    sgemm2_kernel<128><<<grid, 256, 0, st>>>(o1, o2, A2 ? 1 : 0, C, M, N, K, ldc, sC, alpha, beta,
                                            1, nullptr);
    CASCADE_LAUNCHED();
    return cudaGetLastError();
  }
  // few tiles: 64 x 64 tiles and, if there is scratch, K split into slices
  const int64_t tiles64 = (int64_t)((M + 63) / 64) * ((N + 63) / 64) * batch;
  int ks = (int)std::min<int64_t>((2 * sms + tiles64 - 1) / tiles64, std::max(1, K / 64));
  while (ks > 1 && (size_t)ks * batch * M * N > scratch_floats) --ks;
  if (!scratch) ks = 1;
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch * ks);
  sgemm2_kernel<64><<<grid, 256, 0, st>>>(o1, o2, A2 ? 1 : 0, C, M, N, K, ldc, sC, alpha, beta,
                                         ks, scratch);
  CASCADE_LAUNCHED();
  if (ks > 1) {
    const int64_t mn = (int64_t)M * N;
    const int blocks = (int)std::min<int64_t>((mn + 255) / 256, 1024);
    splitk_sum_kernel<<<dim3(blocks, batch), 256, 0, st>>>(scratch, ks, batch, M, N, C, ldc, sC,
                                                          beta);
    CASCADE_LAUNCHED();
  }
  return cudaGetLastError();
}

cudaError_t launch_sgemm(const float* A, const float* B, float* C, int M, int N, int K, int lda,
                         int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC, int batch,
                         float alpha, float beta, bool transA, bool transB, cudaStream_t st) {
  return launch_gemm<float>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, alpha, beta,
                            transA, transB, st);
}

// ----------------------------------------------------------------------------
// Frobenius norm of each of nmat contiguous matrices of `elems` entries.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) frob_kernel(const double* __restrict__ P, int64_t elems,
                                                   double* __restrict__ out) {
  __shared__ double red[8];
  const double* X = P + (int64_t)blockIdx.x * elems;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < elems; i += blockDim.x) s = fma(X[i], X[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = sqrt(t);
  }
}

cudaError_t launch_frob_norms(const double* P, int nmat, int64_t elems, double* out,
                              cudaStream_t st) {
  if (nmat <= 0) return cudaSuccess;
  frob_kernel<<<nmat, 256, 0, st>>>(P, elems, out);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Operand planes: x (FP64) -> (hi, lo) with hi + lo ~ x.
//   BF16 split: hi = RN_bf16(x), lo = RN_bf16(x - hi).
//   FP32 (TF32 pair): hi = RNA_tf32(x), lo = RNA_tf32(x - hi); both are exact TF32
//   values, so the tensor core's use of the top 19 bits does not truncate them.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void split_bf16_kernel(const double* __restrict__ src, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[i];
    const __nv_bfloat16 h = __double2bfloat16(x);
    hi[i] = h;
    lo[i] = __double2bfloat16(x - (double)__bfloat162float(h));
  }
}

__global__ void split_tf32_kernel(const double* __restrict__ src, float* __restrict__ hi,
                                  float* __restrict__ lo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[i];
    const float h = tf32_rna((float)x);
    hi[i] = h;
    lo[i] = tf32_rna((float)(x - (double)h));
  }
}

cudaError_t launch_split_planes(const double* src, void* hi, void* lo, int64_t n, int precision,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (precision == CASCADE_BF16_SPLIT)
    split_bf16_kernel<<<blocks, 256, 0, st>>>(src, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, n);
  else
    split_tf32_kernel<<<blocks, 256, 0, st>>>(src, (float*)hi, (float*)lo, n);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  to_f32_kernel<<<blocks, 256, 0, st>>>(src, dst, n);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace cascade
