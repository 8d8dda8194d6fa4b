// zoh.cu -- zero-order-hold discretisation (§5) on the device, in FP64:
//
//   Abar = exp(delta A),  Bbar = int_0^delta exp(sA) ds B = (delta A)^-1 (exp(delta A) - I) delta B,
//
// both read off E = exp(Z), Z = delta [[A, B], [0, 0]] ((m+p) x (m+p)): Abar is
// E's upper left block, Bbar its upper right block.  The adjoint (gradients to
// A and B) uses the Frechet derivative of the exponential: dZ = L(Z^T, G) with G
// holding (dAbar, dBbar) in those blocks, read off the upper right block of
// exp([[Z^T, G], [0, Z^T]]).
//
// The exponential is the scaling-and-squaring method with a diagonal Pade
// approximant (Higham, SIAM J. Matrix Anal. Appl. 26(4), 2005): Z is scaled by
// 2^-s so that ||Z||_1 <= THETA, r(Z) = q(Z)^-1 p(Z) with
//   p(x) = sum_j b_j x^j,  b_j = (2d - j)! d! / ((2d)! j! (d - j)!),  q(x) = p(-x),
// d = 13, is evaluated from Z^2, Z^4, Z^6 (even part V, odd part U, so p = V + U
// and q = V - U), the system (V - U) R = V + U is solved by Gauss-Jordan
// elimination, and R is squared s times.  THETA = 4: the [d/d] remainder
// (d!)^2 / ((2d)! (2d+1)!) THETA^(2d+1) is below 2e-19 for d = 13.
#include "common.cuh"

#include <math.h>

#include <vector>

namespace cascade {
namespace {

constexpr int PADE_D = 13;
constexpr double THETA = 4.0;

// Z = delta [[A, B], [0, 0]] (transpose: Z^T), n = m + p, per system.
__global__ void zoh_block_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                 const double* __restrict__ delta, double* __restrict__ Z, int m,
                                 int p, int transpose) {
  const int s = blockIdx.y, n = m + p;
  const double dl = delta[s];
  const double* As = A + (int64_t)s * m * m;
  const double* Bs = B + (int64_t)s * m * p;
  double* Zs = Z + (int64_t)s * n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (transpose) { const int t = i; i = j; j = t; }
    double v = 0.0;
    if (i < m) v = j < m ? As[(int64_t)i * m + j] : Bs[(int64_t)i * p + (j - m)];
    Zs[e] = dl * v;
  }
}

// W = [[X, G'], [0, X]] (2n x 2n) with X = Z^T and G' = G / g, where G holds
// (dAbar * scale, dBbar) in its upper blocks and g = max(1, ||G||_1) (written to
// gnorm), so that ||W||_1 <= ||Z^T||_1 + 1.
__global__ void frechet_block_kernel(const double* __restrict__ ZT, const double* __restrict__ dAbar,
                                     const double* __restrict__ dBbar,
                                     const double* __restrict__ scale, double* __restrict__ W,
                                     double* __restrict__ gnorm, int m, int p) {
  const int s = blockIdx.x, n = m + p, n2 = 2 * n;
  const double sc = scale ? scale[s] : 1.0;
  const double* dA = dAbar + (int64_t)s * m * m;
  const double* dB = dBbar + (int64_t)s * m * p;
  __shared__ double red[32];
  __shared__ double s_g;
  // ||G||_1: largest column sum of |G|
  double best = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double c = 0.0;
    for (int i = 0; i < m; ++i)
      c += fabs(j < m ? sc * dA[(int64_t)i * m + j] : dB[(int64_t)i * p + (j - m)]);
    best = fmax(best, c);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) b = fmax(b, red[w]);
    s_g = fmax(1.0, b);
    gnorm[s] = s_g;
  }
  __syncthreads();
  const double ig = 1.0 / s_g;
  const double* X = ZT + (int64_t)s * n * n;
  double* Ws = W + (int64_t)s * n2 * n2;
  for (int64_t e = threadIdx.x; e < (int64_t)n2 * n2; e += blockDim.x) {
    const int i = (int)(e / n2), j = (int)(e % n2);
    double v = 0.0;
    if (i < n && j < n) v = X[(int64_t)i * n + j];
    else if (i >= n && j >= n) v = X[(int64_t)(i - n) * n + (j - n)];
    else if (i < m && j >= n) {
      const int jj = j - n;
      v = ig * (jj < m ? sc * dA[(int64_t)i * m + jj] : dB[(int64_t)i * p + (jj - m)]);
    }
    Ws[e] = v;
  }
}

// Largest column sum (1-norm) and largest row sum (inf-norm) of each n x n matrix.
__global__ void norms_kernel(const double* __restrict__ X, int n, double* __restrict__ n1,
                             double* __restrict__ ninf) {
  const int s = blockIdx.x;
  const double* Xs = X + (int64_t)s * n * n;
  __shared__ double r1[32], r2[32];
  double b1 = 0.0, b2 = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double c = 0.0, r = 0.0;
    for (int i = 0; i < n; ++i) {
      c += fabs(Xs[(int64_t)i * n + j]);
      r += fabs(Xs[(int64_t)j * n + i]);
    }
    b1 = fmax(b1, c);
    b2 = fmax(b2, r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    b1 = fmax(b1, __shfl_down_sync(0xffffffffu, b1, o));
    b2 = fmax(b2, __shfl_down_sync(0xffffffffu, b2, o));
  }
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = b1; r2[threadIdx.x >> 5] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) { a = fmax(a, r1[w]); b = fmax(b, r2[w]); }
    n1[s] = a;
    if (ninf) ninf[s] = b;
  }
}

// X_s *= f_s
__global__ void scale_kernel(double* __restrict__ X, int64_t elems, const double* __restrict__ f) {
  const int s = blockIdx.y;
  const double a = f[s];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < elems;
       e += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)s * elems + e] *= a;
}

// out = c1 X1 + c2 X2 + c3 X3 + c0 I  (+ out if acc), n x n per system
__global__ void lincomb_kernel(double* __restrict__ out, const double* __restrict__ X1, double c1,
                               const double* __restrict__ X2, double c2,
                               const double* __restrict__ X3, double c3, double c0, int n,
                               int acc) {
  const int s = blockIdx.y;
  const int64_t nn = (int64_t)n * n, off = (int64_t)s * nn;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = c1 * X1[off + e] + c2 * X2[off + e] + c3 * X3[off + e];
    if (e / n == e % n) v += c0;
    out[off + e] = acc ? out[off + e] + v : v;
  }
}

// Aug = [V - U | V + U] (n x 2n)
__global__ void pade_system_kernel(const double* __restrict__ U, const double* __restrict__ V,
                                   double* __restrict__ Aug, int n) {
  const int s = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const double u = U[(int64_t)s * nn + e], v = V[(int64_t)s * nn + e];
    double* row = Aug + (int64_t)s * 2 * nn + i * 2 * n;
    row[j] = v - u;
    row[n + j] = v + u;
  }
}

// Gauss-Jordan elimination with partial pivoting on each n x W augmented
// matrix (one block per system): afterwards columns n..W-1 hold the solution.
__global__ void __launch_bounds__(1024) gj_kernel(double* __restrict__ Aug, int n, int W,
                                                  int32_t* singular) {
  extern __shared__ double fac[];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv;
  __shared__ double s_inv;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* T = Aug + (int64_t)blockIdx.x * n * W;
  for (int c = 0; c < n; ++c) {
    double best = -1.0;
    int bi = c;
    for (int i = c + tid; i < n; i += nt) {
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
    for (int j = c + tid; j < W; j += nt) T[(int64_t)c * W + j] *= inv;
    for (int i = tid; i < n; i += nt) fac[i] = (i == c) ? 0.0 : T[(int64_t)i * W + c];
    __syncthreads();
    const int wc = W - c;
    for (int64_t idx = tid; idx < (int64_t)n * wc; idx += nt) {
      const int i = (int)(idx / wc), j = c + (int)(idx % wc);
      const double f = fac[i];
      if (f != 0.0) T[(int64_t)i * W + j] -= f * T[(int64_t)c * W + j];
    }
    __syncthreads();
  }
}

// Out = block (r0, c0) of size rows x cols of each n x n matrix, times f_s (f may be null).
__global__ void block_kernel(const double* __restrict__ X, int n, int r0, int c0, int rows,
                             int cols, double* __restrict__ out, int64_t out_stride,
                             const double* __restrict__ f, double c) {
  const int s = blockIdx.y;
  const double a = c * (f ? f[s] : 1.0);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    out[(int64_t)s * out_stride + e] = a * X[(int64_t)s * n * n + (int64_t)(r0 + i) * n + c0 + j];
  }
}

// Solution columns of Aug (n x 2n) -> R (n x n)
__global__ void take_solution_kernel(const double* __restrict__ Aug, double* __restrict__ R, int n) {
  const int s = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    R[(int64_t)s * nn + e] = Aug[(int64_t)s * 2 * nn + i * 2 * n + n + j];
  }
}

int grid_for(int64_t elems) {
  const int64_t b = (elems + 255) / 256;
  return (int)(b < 1024 ? (b > 0 ? b : 1) : 1024);
}

}  // namespace

size_t expm_scratch_doubles(int n, int ns) { return (size_t)ns * 10 * n * n; }

int expm_squarings(double norm1) {
  if (!(norm1 > THETA)) return 0;
  return (int)ceil(log2(norm1 / THETA));
}

// In place: X_s <- exp(X_s) for ns matrices of n x n.  Each is scaled by
// d_f[s] = 2^-sq[s] first (sq from expm_squarings of its 1-norm; d_f on the
// device) and its Pade value squared sq[s] times.  scratch: expm_scratch_doubles.
cudaError_t expm_batched(double* X, int n, int ns, const std::vector<int>& sq, const double* d_f,
                         double* scratch, int32_t* singular, cudaStream_t st) {
  const int64_t nn = (int64_t)n * n;
  double* Z2 = scratch;
  double* Z4 = Z2 + ns * nn;
  double* Z6 = Z4 + ns * nn;
  double* T1 = Z6 + ns * nn;
  double* U = T1 + ns * nn;
  double* V = U + ns * nn;
  double* Aug = V + ns * nn;       // 2 n^2 per system
  double* R2 = Aug + 2 * ns * nn;  // squaring partner
  // Pade coefficients from b_0 = 1, b_(j+1) = b_j (d - j) / ((2d - j)(j + 1))
  double b[PADE_D + 1];
  b[0] = 1.0;
  for (int j = 0; j < PADE_D; ++j) b[j + 1] = b[j] * (PADE_D - j) / ((2.0 * PADE_D - j) * (j + 1));
  cudaError_t e;
  const dim3 g(grid_for(nn), ns);
  scale_kernel<<<g, 256, 0, st>>>(X, nn, d_f);
  CASCADE_LAUNCHED();
  auto gemm = [&](const double* A, const double* B, double* C) {
    return launch_dgemm(A, B, C, n, n, n, n, n, n, nn, nn, nn, ns, 1.0, 0.0, false, false, st);
  };
  if ((e = gemm(X, X, Z2)) != cudaSuccess) return e;
  if ((e = gemm(Z2, Z2, Z4)) != cudaSuccess) return e;
  if ((e = gemm(Z4, Z2, Z6)) != cudaSuccess) return e;
  // odd part: U = Z (Z6 (b13 Z6 + b11 Z4 + b9 Z2) + b7 Z6 + b5 Z4 + b3 Z2 + b1 I)
  lincomb_kernel<<<g, 256, 0, st>>>(T1, Z6, b[13], Z4, b[11], Z2, b[9], 0.0, n, 0);
  CASCADE_LAUNCHED();
  if ((e = gemm(Z6, T1, U)) != cudaSuccess) return e;
  lincomb_kernel<<<g, 256, 0, st>>>(U, Z6, b[7], Z4, b[5], Z2, b[3], b[1], n, 1);
  CASCADE_LAUNCHED();
  if ((e = gemm(X, U, T1)) != cudaSuccess) return e;   // T1 = U
  // even part: V = Z6 (b12 Z6 + b10 Z4 + b8 Z2) + b6 Z6 + b4 Z4 + b2 Z2 + b0 I
  lincomb_kernel<<<g, 256, 0, st>>>(U, Z6, b[12], Z4, b[10], Z2, b[8], 0.0, n, 0);
  CASCADE_LAUNCHED();
  if ((e = gemm(Z6, U, V)) != cudaSuccess) return e;
  lincomb_kernel<<<g, 256, 0, st>>>(V, Z6, b[6], Z4, b[4], Z2, b[2], b[0], n, 1);
  CASCADE_LAUNCHED();
  // (V - U) R = V + U
  pade_system_kernel<<<g, 256, 0, st>>>(T1, V, Aug, n);
  CASCADE_LAUNCHED();
  const size_t smem = sizeof(double) * (size_t)n;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gj_kernel<<<ns, 1024, smem, st>>>(Aug, n, 2 * n, singular);
  CASCADE_LAUNCHED();
  take_solution_kernel<<<g, 256, 0, st>>>(Aug, X, n);
  CASCADE_LAUNCHED();
  // undo the scaling: square s_s times, system by system
  for (int s = 0; s < ns; ++s) {
    double* a = X + s * nn;
    double* c = R2 + s * nn;
    for (int k = 0; k < sq[s]; ++k) {
      e = launch_dgemm(a, a, c, n, n, n, n, n, n, nn, nn, nn, 1, 1.0, 0.0, false, false, st);
      if (e != cudaSuccess) return e;
      double* t = a; a = c; c = t;
    }
    if (a != X + s * nn) {
      e = cudaMemcpyAsync(X + s * nn, a, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_zoh_block(const double* A, const double* B, const double* delta, double* Z,
                             int m, int p, int ns, bool transpose, cudaStream_t st) {
  const int n = m + p;
  zoh_block_kernel<<<dim3(grid_for((int64_t)n * n), ns), 256, 0, st>>>(A, B, delta, Z, m, p,
                                                                       transpose ? 1 : 0);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_norms(const double* X, int n, int ns, double* n1, double* ninf,
                         cudaStream_t st) {
  norms_kernel<<<ns, 256, 0, st>>>(X, n, n1, ninf);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_frechet_block(const double* ZT, const double* dAbar, const double* dBbar,
                                 const double* scale, double* W, double* gnorm, int m, int p,
                                 int ns, cudaStream_t st) {
  frechet_block_kernel<<<ns, 256, 0, st>>>(ZT, dAbar, dBbar, scale, W, gnorm, m, p);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_block(const double* X, int n, int r0, int c0, int rows, int cols, double* out,
                         int64_t out_stride, const double* f, double c, int ns, cudaStream_t st) {
  block_kernel<<<dim3(grid_for((int64_t)rows * cols), ns), 256, 0, st>>>(X, n, r0, c0, rows, cols,
                                                                         out, out_stride, f, c);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace cascade
