// proj.cu -- the narrow projections around the cascade, as register-tiled
// GEMMs on the CUDA cores (FP32 arithmetic, tensor-core state formats):
//
//   expand   (p or q columns -> m state columns)
//     first stage fused with the input projection (§3, Eq. 3.2 with v^(0) = Bbar u):
//         v^(1)_l = Bbar u_l + (Abar Bbar) u_(l-1)
//     (the work-efficient schedule's first up-sweep level adds the second
//     term on odd l only)
//     adjoint seed of the backward:  W^(N+1)_l = C^T G_l
//   contract (m state columns -> p or q columns)
//     output projection (end of §3):            y_l  = C v_l + D u_l
//     adjoint of the first stage:               du_l = Bbar^T W_l + (Abar Bbar)^T W_(l+1) + D^T G_l
//
// Coefficients are addressed through strides, M(i, j) = M[sys * ss + i * si + j * sj], so the
// same kernels read Bbar [m,p], C [q,m] and D [q,p] as they are stored or transposed.
// One block computes one 128-row tile of one sequence against a 64-column block
// of the result; rows outside the sequence read as zero (x_(-1) = 0, §1).
#include "common.cuh"
#include "formats.cuh"
#include "ptx.cuh"

namespace cascade {
namespace {

constexpr int PBM = 128;   // rows per tile (the tensor-core tile height)

struct Coef {
  const float* M;
  int64_t ss, si, sj;
  __device__ __forceinline__ float at(int sys, int i, int j) const {
    return M[(int64_t)sys * ss + (int64_t)i * si + (int64_t)j * sj];
  }
};

// 8 FP32 values -> (hi, lo) planes of the format at element offset `off`.
template <int FMT>
__device__ __forceinline__ void store8(void* hi, void* lo, int64_t off, const float* v) {
  if constexpr (FMT == FMT_BF16) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      const float2 hf = __bfloat1622float2(hh);
      const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
      hw[j] = *reinterpret_cast<const uint32_t*>(&hh);
      lw[j] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(hi) + off) =
        make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(lo) + off) =
        make_uint4(lw[0], lw[1], lw[2], lw[3]);
  } else {
    float hv[8], lv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      hv[e] = ptx::tf32_rna(v[e]);
      lv[e] = ptx::tf32_rna(v[e] - hv[e]);
    }
    float4* h = reinterpret_cast<float4*>(static_cast<float*>(hi) + off);
    float4* l = reinterpret_cast<float4*>(static_cast<float*>(lo) + off);
    h[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
    h[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
    l[0] = make_float4(lv[0], lv[1], lv[2], lv[3]);
    l[1] = make_float4(lv[4], lv[5], lv[6], lv[7]);
  }
}

// 8 consecutive state entries (hi + lo) as FP32.
template <int FMT>
__device__ __forceinline__ void load8(const void* hi, const void* lo, int64_t off, float* v) {
  if constexpr (FMT == FMT_BF16) {
    const uint4 h = *reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(hi) + off);
    const uint4 l = *reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(lo) + off);
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // a BF16 value is the upper half of the FP32 with the same bits
      v[2 * j] = __uint_as_float(hw[j] << 16) + __uint_as_float(lw[j] << 16);
      v[2 * j + 1] = __uint_as_float(hw[j] & 0xffff0000u) + __uint_as_float(lw[j] & 0xffff0000u);
    }
  } else {
    const float4* h = reinterpret_cast<const float4*>(static_cast<const float*>(hi) + off);
    const float4* l = reinterpret_cast<const float4*>(static_cast<const float*>(lo) + off);
    const float4 h0 = h[0], h1 = h[1], l0 = l[0], l1 = l[1];
    v[0] = h0.x + l0.x; v[1] = h0.y + l0.y; v[2] = h0.z + l0.z; v[3] = h0.w + l0.w;
    v[4] = h1.x + l1.x; v[5] = h1.y + l1.y; v[6] = h1.z + l1.z; v[7] = h1.w + l1.w;
  }
}

// ------------------------------------------------------------------ expand
// out_l[c] = sum_j M1(c, j) X_l[j] (+ sum_j M2(c, j) X_(l-1)[j], on odd l only if
// odd_only),  c < m, j < px.  Thread (cg, rg): columns c0 + 8 cg .. +8, rows
// rg + 32 i (i < 4); tiles start at even l, so l has the parity of rg.
constexpr int EKC = 32;
template <int FMT, bool TWO>
__global__ void __launch_bounds__(256) expand_kernel(const Tile* __restrict__ tiles, int m, int px,
                                                     const float* __restrict__ X, int ldx,
                                                     Coef M1, Coef M2, Bufs out, int buf_mode,
                                                     int buf_fixed, int odd_only) {
  __shared__ float Xs[PBM + 1][EKC + 1];        // row 0: time t0 - 1
  __shared__ __align__(16) float M1s[EKC][64];
  __shared__ __align__(16) float M2s[TWO ? EKC : 1][64];
  const Tile t = tiles[blockIdx.x];
  const int c0 = blockIdx.y * 64;
  const int cg = threadIdx.x & 7, rg = threadIdx.x >> 3;
  const bool second = TWO && (!odd_only || ((t.t0 + rg) & 1) != 0);
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[i][e] = 0.f;
  for (int j0 = 0; j0 < px; j0 += EKC) {
    const int kc = min(EKC, px - j0);
    for (int e = threadIdx.x; e < (PBM + 1) * EKC; e += 256) {
      const int r = e / EKC, jj = e - r * EKC;
      const int tm = t.t0 - 1 + r;
      float v = 0.f;
      if (jj < kc && tm >= 0 && tm < t.len) v = X[(t.seq_row0 + tm) * ldx + j0 + jj];
      Xs[r][jj] = v;
    }
    for (int e = threadIdx.x; e < EKC * 64; e += 256) {
      const int jj = e >> 6, cc = e & 63;
      const bool ok = jj < kc && c0 + cc < m;
      M1s[jj][cc] = ok ? M1.at(t.sys, c0 + cc, j0 + jj) : 0.f;
      if (TWO) M2s[jj][cc] = ok ? M2.at(t.sys, c0 + cc, j0 + jj) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kc; ++jj) {
      float b1[8], b2[8];
      const float4 p0 = *reinterpret_cast<const float4*>(&M1s[jj][cg * 8]);
      const float4 p1 = *reinterpret_cast<const float4*>(&M1s[jj][cg * 8 + 4]);
      b1[0] = p0.x; b1[1] = p0.y; b1[2] = p0.z; b1[3] = p0.w;
      b1[4] = p1.x; b1[5] = p1.y; b1[6] = p1.z; b1[7] = p1.w;
      if (TWO) {
        const float4 q0 = *reinterpret_cast<const float4*>(&M2s[jj][cg * 8]);
        const float4 q1 = *reinterpret_cast<const float4*>(&M2s[jj][cg * 8 + 4]);
        b2[0] = q0.x; b2[1] = q0.y; b2[2] = q0.z; b2[3] = q0.w;
        b2[4] = q1.x; b2[5] = q1.y; b2[6] = q1.z; b2[7] = q1.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = rg + 32 * i;
        const float x1 = Xs[r + 1][jj];
        const float x0 = second ? Xs[r][jj] : 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          acc[i][e] = fmaf(b1[e], x1, acc[i][e]);
          if (TWO) acc[i][e] = fmaf(b2[e], x0, acc[i][e]);
        }
      }
    }
    __syncthreads();
  }
  const int c = c0 + cg * 8;
  if (c >= m) return;
  const int b = buf_mode ? ((t.flags + 1) & 1) : buf_fixed;
  void* hi = out.hi(b);
  void* lo = out.lo(b);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = rg + 32 * i;
    if (t.t0 + r >= t.len) continue;
    if (odd_only == 2 && ((t.t0 + r) & 1) == 0 && t.t0 + r != 0) continue;   // formed later
    store8<FMT>(hi, lo, (t.seq_row0 + t.t0 + r) * (int64_t)m + c, acc[i]);
  }
}

// ------------------------------------------------------------------ contract
// out_l[j] = sum_c M1(j, c) V_l[c] (+ sum_c M2(j, c) V_(l+1)[c]) + sum_i M3(j, i) X_l[i],
// j < nout, c < m, i < px.  The K loop runs over the m state columns, then over
// the px dense columns.  Thread (cg, rg): rows 4 rg .. +4, columns j0 + CT cg .. +CT.
constexpr int CKC = 16;
template <int FMT, bool TWO, int CT>
__global__ void __launch_bounds__(256) contract_kernel(const Tile* __restrict__ tiles, int m,
                                                       int nout, Bufs V, int buf_mode,
                                                       int buf_fixed, Coef M1, Coef M2, Coef M3,
                                                       const float* __restrict__ X, int px,
                                                       float* __restrict__ out) {
  constexpr int QB = 8 * CT;
  __shared__ __align__(16) float Vs[CKC][PBM + 4];
  __shared__ __align__(16) float V2s[TWO ? CKC : 1][PBM + 4];
  __shared__ __align__(16) float M1s[CKC][QB];
  __shared__ __align__(16) float M2s[TWO ? CKC : 1][QB];
  const Tile t = tiles[blockIdx.x];
  const int j0 = blockIdx.y * QB;
  const int cg = threadIdx.x & 7, rg = threadIdx.x >> 3;
  const int b = buf_mode ? t.fbuf : buf_fixed;
  const void* vh = V.hi(b);
  const void* vl = V.lo(b);
  float acc[4][CT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int e = 0; e < CT; ++e) acc[i][e] = 0.f;
  // loader: thread -> (row lr, 8 columns lc8) of the 128 x 16 chunk
  const int lr = threadIdx.x >> 1, lc8 = (threadIdx.x & 1) * 8;
  const int tl = t.t0 + lr;
  const int64_t lrow = t.seq_row0 + tl;
  const int nk = m + px;
  for (int k0 = 0; k0 < nk; k0 += CKC) {
    const bool dense = k0 >= m;            // m % 16 == 0: a chunk is all V or all X
    const int kd = k0 - m;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = 0.f;
    if (tl < t.len) {
      if (!dense) {
        load8<FMT>(vh, vl, lrow * m + k0 + lc8, v);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (kd + lc8 + e < px) v[e] = X[lrow * px + kd + lc8 + e];
      }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) Vs[lc8 + e][lr] = v[e];
    const bool two = TWO && !dense;
    if (two) {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
      if (tl + 1 < t.len) load8<FMT>(vh, vl, (lrow + 1) * m + k0 + lc8, v);
#pragma unroll
      for (int e = 0; e < 8; ++e) V2s[lc8 + e][lr] = v[e];
    }
    for (int e = threadIdx.x; e < CKC * QB; e += 256) {
      const int kk = e / QB, jj = e - kk * QB;
      const bool ok = j0 + jj < nout;
      if (!dense) {
        M1s[kk][jj] = ok ? M1.at(t.sys, j0 + jj, k0 + kk) : 0.f;
        if (TWO) M2s[kk][jj] = ok ? M2.at(t.sys, j0 + jj, k0 + kk) : 0.f;
      } else {
        M1s[kk][jj] = (ok && kd + kk < px) ? M3.at(t.sys, j0 + jj, kd + kk) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < CKC; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&Vs[kk][rg * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      float mv[CT];
#pragma unroll
      for (int e = 0; e < CT; ++e) mv[e] = M1s[kk][cg * CT + e];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int e = 0; e < CT; ++e) acc[i][e] = fmaf(av[i], mv[e], acc[i][e]);
      if (two) {
        const float4 a2 = *reinterpret_cast<const float4*>(&V2s[kk][rg * 4]);
        const float av2[4] = {a2.x, a2.y, a2.z, a2.w};
#pragma unroll
        for (int e = 0; e < CT; ++e) mv[e] = M2s[kk][cg * CT + e];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int e = 0; e < CT; ++e) acc[i][e] = fmaf(av2[i], mv[e], acc[i][e]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = rg * 4 + i;
    if (t.t0 + r >= t.len) continue;
    const int64_t row = t.seq_row0 + t.t0 + r;
#pragma unroll
    for (int e = 0; e < CT; ++e) {
      const int j = j0 + cg * CT + e;
      if (j < nout) out[row * nout + j] = acc[i][e];
    }
  }
}

// ------------------------------------------------------------------ narrow forms
// With px (expand) or nout (contract) of a few columns the GEMM tiles above are
// mostly padding; these stream the state rows instead.  Coefficients sit in
// shared memory as [j][c] (m * width <= THIN_ELEMS floats per matrix).
constexpr int THIN_ELEMS = 4096;

// Shared-memory position of coefficient (j, c): column c = 8 g + 4 h + t is
// stored so that the 32 threads reading the 4-column half h of consecutive
// groups g touch 512 consecutive bytes (no bank conflicts):
//   j * stride + (g / 32) * 256 + h * 128 + (g % 32) * 4 + t,  stride = m rounded up to 256.
__device__ __forceinline__ int thin_idx(int j, int c, int stride) {
  const int g = c >> 3, h = (c >> 2) & 1, t = c & 3;
  return j * stride + (g >> 5) * 256 + h * 128 + (g & 31) * 4 + t;
}
__host__ __device__ __forceinline__ int thin_stride(int m) { return (m + 255) & ~255; }

// expand: v[l, c] = sum_j M1[c, j] X[l, j] + [second term] sum_j M2[c, j] X[l - 1, j]
// over the rows of each tile.  Persistent: block b takes the contiguous tiles
// [b * per, (b + 1) * per), so the coefficients are reloaded only when the
// system changes.  Thread layout: column group g = tid % G (8 columns,
// G = m / 8), row phase tid / G, RPI = 256 / G rows per pass; with PXR = px = 1
// a thread's coefficients stay in registers, otherwise they are read from
// shared memory in the [j][c] layout above.  The next tile's X rows are fetched
// into registers while the current tile is stored (its record one tile earlier).
constexpr int XPF = ((PBM + 1) * 8 + 255) / 256;   // X values per thread (px <= 8)
constexpr int EXPAND_BLOCKS_PER_SM = 4;

template <int FMT, bool TWO, int PXR>
__global__ void __launch_bounds__(256, EXPAND_BLOCKS_PER_SM)
    expand_thin_kernel(const Tile* __restrict__ tiles, int ntiles, int per, int m, int px,
                       const float* __restrict__ X, int ldx, Coef M1, Coef M2, Bufs out,
                       int buf_mode, int buf_fixed, int odd_only) {
  extern __shared__ __align__(16) float esm[];
  const int PX = PXR > 0 ? PXR : px;
  const int stride = thin_stride(m);
  float* Xs = esm;                           // [(PBM + 1) * PX], row 0: time t0 - 1
  float* M1s = esm + (PBM + 1) * 8;          // [PX][stride] (PXR == 0)
  float* M2s = M1s + PX * stride;
  const int tid = threadIdx.x;
  const int G = m >> 3, RPI = 256 / G;
  const int g = tid % G, rph = tid / G;
  const int c0 = g * 8;
  const bool active = rph < RPI;
  const int nx = (PBM + 1) * PX;
  const int tb = blockIdx.x * per, te = min(ntiles, tb + per);
  float m1[PXR > 0 ? PXR : 1][8], m2[PXR > 0 && TWO ? PXR : 1][8];
  float xr[XPF];
  auto fetch = [&](const Tile& t) {
#pragma unroll
    for (int i = 0; i < XPF; ++i) {
      const int e = tid + i * 256;
      float v = 0.f;
      if (e < nx) {
        const int r = e / PX, j = e - r * PX;
        const int l = t.t0 - 1 + r;
        if (l >= 0 && l < t.len) v = __ldg(X + (t.seq_row0 + l) * ldx + j);
      }
      xr[i] = v;
    }
  };
  // Tile records run two ahead of the stores, X rows one ahead.
  Tile tnext{};
  if (tb < te) {
    fetch(tiles[tb]);
    tnext = tiles[tb + 1 < te ? tb + 1 : tb];
  }
  int cur_sys = -1;
  for (int ti = tb; ti < te; ++ti) {
    const Tile t = tiles[ti];
    __syncthreads();   // every read of Xs (and M1s, M2s) for the previous tile is done
#pragma unroll
    for (int i = 0; i < XPF; ++i)
      if (tid + i * 256 < nx) Xs[tid + i * 256] = xr[i];
    if (t.sys != cur_sys) {   // block-uniform
      cur_sys = t.sys;
      if constexpr (PXR == 0) {
        for (int e = tid; e < PX * m; e += 256) {
          const int j = e / m, c = e - j * m;
          M1s[thin_idx(j, c, stride)] = M1.at(t.sys, c, j);
          if (TWO) M2s[thin_idx(j, c, stride)] = M2.at(t.sys, c, j);
        }
      } else if (active) {
#pragma unroll
        for (int j = 0; j < PXR; ++j)
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            m1[j][e] = M1.at(t.sys, c0 + e, j);
            if (TWO) m2[j][e] = M2.at(t.sys, c0 + e, j);
          }
      }
    }
    __syncthreads();
    if (ti + 1 < te) {
      fetch(tnext);
      tnext = tiles[ti + 2 < te ? ti + 2 : ti + 1];
    }
    if (!active) continue;
    const int b = buf_mode ? ((t.flags + 1) & 1) : buf_fixed;
    void* hi = out.hi(b);
    void* lo = out.lo(b);
    const int rows = min(PBM, t.len - t.t0);
#pragma unroll 2
    for (int r = rph; r < rows; r += RPI) {
      const int l = t.t0 + r;
      const bool second = TWO && l >= 1 && (!odd_only || (l & 1));
      float acc[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = 0.f;
      for (int j = 0; j < PX; ++j) {
        const float x1 = Xs[(r + 1) * PX + j];
        const float x0 = second ? Xs[r * PX + j] : 0.f;
        if constexpr (PXR > 0) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            acc[e] = fmaf(m1[j][e], x1, acc[e]);
            if (TWO) acc[e] = fmaf(m2[j][e], x0, acc[e]);
          }
        } else {
          const float4 a0 = *reinterpret_cast<const float4*>(&M1s[thin_idx(j, c0, stride)]);
          const float4 a1 = *reinterpret_cast<const float4*>(&M1s[thin_idx(j, c0 + 4, stride)]);
          acc[0] = fmaf(a0.x, x1, acc[0]); acc[1] = fmaf(a0.y, x1, acc[1]);
          acc[2] = fmaf(a0.z, x1, acc[2]); acc[3] = fmaf(a0.w, x1, acc[3]);
          acc[4] = fmaf(a1.x, x1, acc[4]); acc[5] = fmaf(a1.y, x1, acc[5]);
          acc[6] = fmaf(a1.z, x1, acc[6]); acc[7] = fmaf(a1.w, x1, acc[7]);
          if (TWO) {
            const float4 b0 = *reinterpret_cast<const float4*>(&M2s[thin_idx(j, c0, stride)]);
            const float4 b1 = *reinterpret_cast<const float4*>(&M2s[thin_idx(j, c0 + 4, stride)]);
            acc[0] = fmaf(b0.x, x0, acc[0]); acc[1] = fmaf(b0.y, x0, acc[1]);
            acc[2] = fmaf(b0.z, x0, acc[2]); acc[3] = fmaf(b0.w, x0, acc[3]);
            acc[4] = fmaf(b1.x, x0, acc[4]); acc[5] = fmaf(b1.y, x0, acc[5]);
            acc[6] = fmaf(b1.z, x0, acc[6]); acc[7] = fmaf(b1.w, x0, acc[7]);
          }
        }
      }
      if (odd_only == 2 && !(l & 1) && l != 0) continue;   // formed later from u
      store8<FMT>(hi, lo, (t.seq_row0 + l) * (int64_t)m + c0, acc);
    }
  }
}

// contract: each warp walks 16 consecutive rows of the tile, lanes over 8-column
// groups (NCH groups per lane, m <= 256 NCH), then a warp reduction per output
// column.  With the shifted term, row l+1 is loaded once and serves as the
// next row of l and then as the row itself.
template <int FMT, bool TWO, int NCH, int QT>
__global__ void __launch_bounds__(256) contract_thin_kernel(const Tile* __restrict__ tiles, int m,
                                                            int nout, Bufs V, int buf_mode,
                                                            int buf_fixed, Coef M1, Coef M2,
                                                            Coef M3, const float* __restrict__ X,
                                                            int px, float* __restrict__ out) {
  // nout <= QT (1, 2 or 4)
  __shared__ __align__(16) float M1s[THIN_ELEMS];
  __shared__ __align__(16) float M2s[TWO ? THIN_ELEMS : 4];
  const Tile t = tiles[blockIdx.x];
  const int stride = thin_stride(m);
  for (int e = threadIdx.x; e < nout * m; e += 256) {
    const int j = e / m, c = e - j * m;
    M1s[thin_idx(j, c, stride)] = M1.at(t.sys, j, c);
    if (TWO) M2s[thin_idx(j, c, stride)] = M2.at(t.sys, j, c);
  }
  __syncthreads();
  const int b = buf_mode ? t.fbuf : buf_fixed;
  const void* vh = V.hi(b);
  const void* vl = V.lo(b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = min(PBM, t.len - t.t0);
  const int rbeg = warp * 16, rend = min(rows, rbeg + 16);
  auto load_row = [&](int r, float (&v)[NCH][8]) {
    const int64_t row = t.seq_row0 + t.t0 + r;
#pragma unroll
    for (int ci = 0; ci < NCH; ++ci) {
      const int c0 = lane * 8 + ci * 256;
      if (c0 < m && r < t.len - t.t0) {
        load8<FMT>(vh, vl, row * (int64_t)m + c0, v[ci]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[ci][e] = 0.f;
      }
    }
  };
  // rows in register blocks of RB (RB + 1 rows loaded with the shifted term; the
  // last one is carried into the next block)
  constexpr int RB = NCH >= 4 ? 1 : 4 / NCH;
  constexpr int NV = RB + (TWO ? 1 : 0);
  float v[NV][NCH][8];
  bool have0 = false;
  for (int r0 = rbeg; r0 < rend; r0 += RB) {
#pragma unroll
    for (int u = 0; u < NV; ++u)
      if (!(u == 0 && have0)) load_row(r0 + u, v[u]);
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = r0 + u;
      if (r >= rend) break;
      float acc[QT];
#pragma unroll
      for (int j = 0; j < QT; ++j) {
        float sj = 0.f;
        if (j < nout) {
#pragma unroll
          for (int ci = 0; ci < NCH; ++ci) {
            const int c0 = lane * 8 + ci * 256;
            if (c0 >= m) continue;
            const float4 a0 = *reinterpret_cast<const float4*>(&M1s[thin_idx(j, c0, stride)]);
            const float4 a1 = *reinterpret_cast<const float4*>(&M1s[thin_idx(j, c0 + 4, stride)]);
            const float w1[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) sj = fmaf(w1[e], v[u][ci][e], sj);
            if (TWO) {
              const float4 b0 = *reinterpret_cast<const float4*>(&M2s[thin_idx(j, c0, stride)]);
              const float4 b1 =
                  *reinterpret_cast<const float4*>(&M2s[thin_idx(j, c0 + 4, stride)]);
              const float w2[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
              for (int e = 0; e < 8; ++e) sj = fmaf(w2[e], v[u + (TWO ? 1 : 0)][ci][e], sj);
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
        acc[j] = sj;
      }
      if (lane < nout) {
        const int64_t row = t.seq_row0 + t.t0 + r;
        float sv = 0.f;
#pragma unroll
        for (int j = 0; j < QT; ++j)
          if (j == lane) sv = acc[j];
        for (int i = 0; i < px; ++i) sv = fmaf(M3.at(t.sys, lane, i), __ldg(X + row * px + i), sv);
        out[row * nout + lane] = sv;
      }
    }
    if (TWO) {   // row r0 + RB is the first row of the next block
#pragma unroll
      for (int ci = 0; ci < NCH; ++ci)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[0][ci][e] = v[NV - 1][ci][e];
      have0 = true;
    }
  }
}

template <int FMT, bool TWO>
cudaError_t contract_dispatch(const Tile* tiles, int ntiles, int m, int nout, const Bufs& V,
                              int buf_mode, int buf_fixed, const Coef& M1, const Coef& M2,
                              const Coef& M3, const float* X, int px, float* out,
                              cudaStream_t st) {
  if (nout <= 4 && thin_stride(m) * nout <= THIN_ELEMS && m <= 1024) {
    const int nch = (m + 255) / 256;
#define CASCADE_CTHIN(NC, QC)                                                                 \
  contract_thin_kernel<FMT, TWO, NC, QC><<<ntiles, 256, 0, st>>>(tiles, m, nout, V, buf_mode,  \
                                                                 buf_fixed, M1, M2, M3, X, px, out)
#define CASCADE_CTHIN_Q(NC)          \
  if (nout == 1) CASCADE_CTHIN(NC, 1); \
  else if (nout == 2) CASCADE_CTHIN(NC, 2); \
  else CASCADE_CTHIN(NC, 4)
    if (nch == 1) { CASCADE_CTHIN_Q(1); }
    else if (nch == 2) { CASCADE_CTHIN_Q(2); }
    else { CASCADE_CTHIN_Q(4); }
#undef CASCADE_CTHIN_Q
#undef CASCADE_CTHIN
    CASCADE_LAUNCHED();
    return cudaGetLastError();
  }
  const int ct = nout <= 8 ? 1 : nout <= 16 ? 2 : nout <= 32 ? 4 : 8;
  dim3 grid(ntiles, (nout + 8 * ct - 1) / (8 * ct));
#define CASCADE_CONTRACT(CTV)                                                                 \
  contract_kernel<FMT, TWO, CTV><<<grid, 256, 0, st>>>(tiles, m, nout, V, buf_mode, buf_fixed, \
                                                       M1, M2, M3, X, px, out)
  switch (ct) {
    case 1: CASCADE_CONTRACT(1); break;
    case 2: CASCADE_CONTRACT(2); break;
    case 4: CASCADE_CONTRACT(4); break;
    default: CASCADE_CONTRACT(8);
  }
#undef CASCADE_CONTRACT
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

template <bool TWO>
cudaError_t expand_dispatch(int precision, int nsms, const Tile* tiles, int ntiles, int m, int px,
                            const float* X, int ldx, const Coef& M1, const Coef& M2,
                            const Bufs& out, int buf_mode, int buf_fixed, int odd_only,
                            cudaStream_t st) {
  if (px <= 8 && thin_stride(m) * px <= THIN_ELEMS && m / 8 <= 256) {
    const int want = (nsms > 0 ? nsms : 1) * EXPAND_BLOCKS_PER_SM;
    const int per = (ntiles + want - 1) / want;
    const int grid = (ntiles + per - 1) / per;
    const size_t coef = px == 1 ? 0 : (TWO ? 2 : 1) * (size_t)px * thin_stride(m);
    const size_t smem = sizeof(float) * ((size_t)(PBM + 1) * 8 + coef);
#define CASCADE_ETHIN(F, R)                                                                    \
  expand_thin_kernel<F, TWO, R><<<grid, 256, smem, st>>>(tiles, ntiles, per, m, px, X, ldx, M1, \
                                                         M2, out, buf_mode, buf_fixed, odd_only)
    if (precision == CASCADE_BF16_SPLIT) {
      if (px == 1) CASCADE_ETHIN(FMT_BF16, 1);
      else CASCADE_ETHIN(FMT_BF16, 0);
    } else {
      if (px == 1) CASCADE_ETHIN(FMT_F32, 1);
      else CASCADE_ETHIN(FMT_F32, 0);
    }
#undef CASCADE_ETHIN
    CASCADE_LAUNCHED();
    return cudaGetLastError();
  }
  dim3 grid(ntiles, (m + 63) / 64);
  if (precision == CASCADE_BF16_SPLIT)
    expand_kernel<FMT_BF16, TWO><<<grid, 256, 0, st>>>(tiles, m, px, X, ldx, M1, M2, out,
                                                      buf_mode, buf_fixed, odd_only);
  else
    expand_kernel<FMT_F32, TWO><<<grid, 256, 0, st>>>(tiles, m, px, X, ldx, M1, M2, out, buf_mode,
                                                     buf_fixed, odd_only);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

// y = C v + D u for listed rows: one warp per row, lanes over 8-column groups.
template <int FMT>
__global__ void __launch_bounds__(256) rows_output_kernel(const int64_t* __restrict__ rows,
                                                          const int32_t* __restrict__ row_sys,
                                                          int nrows, int m, int q, int px,
                                                          Bufs V, int buf, Coef C, Coef D,
                                                          const float* __restrict__ u,
                                                          float* __restrict__ y) {
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= nrows) return;
  const int64_t row = rows[gw];
  const int s = row_sys[gw];
  for (int j = 0; j < q; ++j) {
    float acc = 0.f;
    for (int c0 = lane * 8; c0 < m; c0 += 256) {
      float v[8];
      load8<FMT>(V.hi(buf), V.lo(buf), row * (int64_t)m + c0, v);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc = fmaf(C.at(s, j, c0 + e), v[e], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      for (int i = 0; i < px; ++i) acc = fmaf(D.at(s, j, i), u[row * px + i], acc);
      y[row * q + j] = acc;
    }
  }
}

}  // namespace

bool proj_supported(const Plan& p) {
  return p.d.precision != CASCADE_FP64 && p.d.m % 16 == 0 && tile_rows(p) == PBM;
}

// v^(1) = Bbar u_l + (Abar Bbar) u_(l-1) into state buffer `buf` (first stage);
// odd_mode 1: the second term on odd l only (first up-sweep level); 2: as 1,
// and of the even rows only row 0 is stored (the last down-sweep level forms
// the others from u).
cudaError_t launch_proj_stage0(const Plan& p, const float* u, const Bufs& V, int buf,
                               int odd_mode, cudaStream_t st) {
  if (p.n_stage0_tiles == 0) return cudaSuccess;
  const int m = p.d.m, pp = p.d.p;
  const Coef B{p.Bbar32, (int64_t)m * pp, pp, 1};     // Bbar [m, p]: (c, j)
  const Coef AB{p.ABbar32, (int64_t)m * pp, pp, 1};
  return expand_dispatch<true>(p.d.precision, p.num_sms, p.d_stage0_tiles, p.n_stage0_tiles, m,
                               pp, u, pp, B, AB, V, 0, buf, odd_mode, st);
}

// W^(N_i+1) = C^T G into adjoint buffer (N_i + 1) & 1 of every tile.
cudaError_t launch_proj_adj_init(const Plan& p, const float* G, const Bufs& W, cudaStream_t st) {
  if (p.n_all_tiles == 0) return cudaSuccess;
  const int m = p.d.m, q = p.d.q;
  const Coef Ct{p.C32, (int64_t)q * m, 1, m};          // C [q, m]: (c, j) = C[j][c]
  return expand_dispatch<false>(p.d.precision, p.num_sms, p.d_all_tiles, p.n_all_tiles, m, q, G,
                                q, Ct, Ct, W, 1, 0, 0, st);
}

// y = C v + D u for the tiles whose output was not fused (state buffer tile.fbuf).
cudaError_t launch_proj_output(const Plan& p, const float* u, float* y, const Bufs& V,
                               cudaStream_t st) {
  if (p.n_out_tiles == 0) return cudaSuccess;
  const int m = p.d.m, pp = p.d.p, q = p.d.q;
  const Coef C{p.C32, (int64_t)q * m, m, 1};           // (j, c)
  const Coef D{p.D32, (int64_t)q * pp, pp, 1};         // (j, i)
  if (p.d.precision == CASCADE_BF16_SPLIT)
    return contract_dispatch<FMT_BF16, false>(p.d_out_tiles, p.n_out_tiles, m, q, V, 1, 0, C, C, D,
                                              u, pp, y, st);
  return contract_dispatch<FMT_F32, false>(p.d_out_tiles, p.n_out_tiles, m, q, V, 1, 0, C, C, D, u,
                                           pp, y, st);
}

// du = Bbar^T W_l + (Abar Bbar)^T W_(l+1) + D^T G_l with W^(1) in adjoint buffer `wbuf`.
cudaError_t launch_proj_du(const Plan& p, const float* G, const Bufs& W, int wbuf, float* du,
                           cudaStream_t st) {
  if (p.n_all_tiles == 0) return cudaSuccess;
  const int m = p.d.m, pp = p.d.p, q = p.d.q;
  const Coef Bt{p.Bbar32, (int64_t)m * pp, 1, pp};     // (j, c) = Bbar[c][j]
  const Coef ABt{p.ABbar32, (int64_t)m * pp, 1, pp};
  const Coef Dt{p.D32, (int64_t)q * pp, 1, pp};        // (j, i) = D[i][j]
  if (p.d.precision == CASCADE_BF16_SPLIT)
    return contract_dispatch<FMT_BF16, true>(p.d_all_tiles, p.n_all_tiles, m, pp, W, 0, wbuf, Bt,
                                             ABt, Dt, G, q, du, st);
  return contract_dispatch<FMT_F32, true>(p.d_all_tiles, p.n_all_tiles, m, pp, W, 0, wbuf, Bt, ABt,
                                          Dt, G, q, du, st);
}

// y = C v + D u for an explicit list of rows (state buffer `buf`).
cudaError_t launch_proj_rows_output(const Plan& p, const int64_t* rows, int nrows,
                                    const int32_t* row_sys, const float* u, float* y,
                                    const Bufs& V, int buf, cudaStream_t st) {
  if (nrows == 0) return cudaSuccess;
  const int m = p.d.m, pp = p.d.p, q = p.d.q;
  const Coef C{p.C32, (int64_t)q * m, m, 1};
  const Coef D{p.D32, (int64_t)q * pp, pp, 1};
  const int blocks = (nrows * 32 + 255) / 256;
  if (p.d.precision == CASCADE_BF16_SPLIT)
    rows_output_kernel<FMT_BF16><<<blocks, 256, 0, st>>>(rows, row_sys, nrows, m, q, pp, V, buf, C,
                                                        D, u, y);
  else
    rows_output_kernel<FMT_F32><<<blocks, 256, 0, st>>>(rows, row_sys, nrows, m, q, pp, V, buf, C, D,
                                                       u, y);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace cascade
