// backward.cu -- kernels of the reverse-mode derivative of the cascade.
//
// Forward (§3): v^(0)_l = Bbar u_l; v^(k+1)_l = v^(k)_l + P_k v^(k)_(l-s_k)
// (s_k = 2^k, zero source before the sequence start); y_l = C v^(N+1)_l + D u_l;
// P_0 = Abar, P_(k+1) = P_k P_k.  With G = dL/dy the adjoint runs the stages
// backwards with the transposed powers and the reversed shift:
//
//   W^(N+1)_l = C^T G_l,
//   W^(k)_l   = W^(k+1)_l + P_k^T W^(k+1)_(l+s_k)      (zero source past the end),
//   dP_k      = sum_l W^(k+1)_l v^(k)_(l-s_k)^T,
//   dC = sum_l G_l v^(N+1)_l^T,  dD = sum_l G_l u_l^T.
//
// The first stage is fused with the input projection in the forward
// (v^(1)_l = Bbar u_l + Abar Bbar u_(l-1)), so its adjoint is fused too:
//
//   du_l   = Bbar^T W^(1)_l + (Abar Bbar)^T W^(1)_(l+1) + D^T G_l,
//   R1     = sum_l W^(1)_l u_l^T,   R2 = sum_l W^(1)_l u_(l-1)^T,
//   dBbar  = R1 + Abar^T R2,        dP_0 += R2 Bbar^T.
//
// This file holds the element-wise and reduction kernels; the adjoint stages
// themselves reuse the forward stage kernels in reverse mode, and the
// squaring-chain and discretisation adjoints are FP64 GEMMs (api.cu).
//
// Reductions over time are split-K: each block sums one chunk of tiles of one
// system into a partial, and a second kernel adds the partials of each system
// in chunk order in FP64, so results are deterministic.
#include "common.cuh"
#include "formats.cuh"

#include <algorithm>

namespace cascade {
namespace {

template <int FMT>
__device__ __forceinline__ typename Acc<FMT>::type src_get(const TSrc& s, const Tile& t,
                                                           int64_t row, int col, int m) {
  typedef typename Acc<FMT>::type A;
  if (s.kind == 1) return (A) static_cast<const float*>(s.dense)[row * s.ld + col];
  if (s.kind == 2) return (A) static_cast<const double*>(s.dense)[row * s.ld + col];
  const int b = s.buf_mode ? t.fbuf : s.buf_fixed;
  return load_elem<FMT>(s.bufs.hi(b), s.bufs.lo(b), row * m + col);
}

// partial[chunk][i][j] = sum over the chunk's rows l (l >= shift) of X[l][i] Y[l - shift][j].
// Block = one 64 x 64 output block of one chunk; 256 threads, 4 x 4 outputs each.
template <int FMT, typename ACC>
__global__ void __launch_bounds__(256) treduce_kernel(const Tile* __restrict__ tiles,
                                                      const int32_t* __restrict__ chunks, int BM,
                                                      int m, TSrc X, int a, TSrc Y, int b, int shift,
                                                      ACC* __restrict__ partial) {
  __shared__ ACC xs[16][65];
  __shared__ ACC ys[16][65];
  const int c = blockIdx.z;
  const int first = chunks[3 * c], count = chunks[3 * c + 1];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  ACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int ti = first; ti < first + count; ++ti) {
    const Tile t = tiles[ti];
    const int rows = min(BM, t.len - t.t0);
    for (int r0 = 0; r0 < rows; r0 += 16) {
      for (int e = threadIdx.x; e < 16 * 64; e += 256) {
        const int rr = e >> 6, col = e & 63;
        const int l = t.t0 + r0 + rr;
        const bool ok = (r0 + rr < rows) && l >= shift;
        const int64_t row = t.seq_row0 + l;
        xs[rr][col] = (ok && i0 + col < a) ? (ACC)src_get<FMT>(X, t, row, i0 + col, m) : (ACC)0;
        ys[rr][col] = (ok && j0 + col < b) ? (ACC)src_get<FMT>(Y, t, row - shift, j0 + col, m)
                                           : (ACC)0;
      }
      __syncthreads();
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        ACC xv[4], yv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = xs[rr][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) yv[j] = ys[rr][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], yv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  ACC* out = partial + (int64_t)c * a * b;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + ty + 16 * i;
    if (gi >= a) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tx + 16 * j;
      if (gj < b) out[(int64_t)gi * b + gj] = acc[i][j];
    }
  }
}

// out[s][e] (+)= sum over the chunks of system s, in order, of partial[chunk][e].
// A chunk's partial may hold several outputs back to back (seg elements each);
// output h of system s starts at out + h * seg_stride + s * out_sys_stride.
template <typename ACC, typename OUT>
__global__ void reduce_partials_kernel(const ACC* __restrict__ partial,
                                       const int32_t* __restrict__ sys_begin, int64_t elems,
                                       OUT* __restrict__ out, int64_t out_sys_stride,
                                       int64_t seg, int64_t seg_stride, int accumulate) {
  const int s = blockIdx.y;
  const int c0 = sys_begin[s], c1 = sys_begin[s + 1];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    OUT v = 0;
    for (int c = c0; c < c1; ++c) v += (OUT)partial[(int64_t)c * elems + e];
    const int64_t h = e / seg;
    OUT* o = out + h * seg_stride + (int64_t)s * out_sys_stride + (e - h * seg);
    *o = accumulate ? *o + v : v;
  }
}

// The same sum over FP32 partials, four consecutive elements per thread
// (elems % 4 == 0) and four chunks' loads in flight per step; the additions
// keep the chunk order, so the result is the scalar kernel's bit for bit.
template <typename OUT>
__global__ void reduce_partials4_kernel(const float* __restrict__ partial,
                                        const int32_t* __restrict__ sys_begin, int64_t elems,
                                        OUT* __restrict__ out, int64_t out_sys_stride,
                                        int64_t seg, int64_t seg_stride, int accumulate) {
  const int s = blockIdx.y;
  const int c0 = sys_begin[s], c1 = sys_begin[s + 1];
  const int64_t n4 = elems >> 2;
  const float4* p4 = reinterpret_cast<const float4*>(partial);
  for (int64_t e4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e4 < n4;
       e4 += (int64_t)gridDim.x * blockDim.x) {
    OUT v[4] = {0, 0, 0, 0};
    int c = c0;
    for (; c + 4 <= c1; c += 4) {
      float4 a[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) a[h] = __ldg(p4 + (int64_t)(c + h) * n4 + e4);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        v[0] += (OUT)a[h].x;
        v[1] += (OUT)a[h].y;
        v[2] += (OUT)a[h].z;
        v[3] += (OUT)a[h].w;
      }
    }
    for (; c < c1; ++c) {
      const float4 a = __ldg(p4 + (int64_t)c * n4 + e4);
      v[0] += (OUT)a.x;
      v[1] += (OUT)a.y;
      v[2] += (OUT)a.z;
      v[3] += (OUT)a.w;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t e = 4 * e4 + j;
      const int64_t h = e / seg;
      OUT* o = out + h * seg_stride + (int64_t)s * out_sys_stride + (e - h * seg);
      *o = accumulate ? *o + v[j] : v[j];
    }
  }
}

// With few systems x elements the sum above has too little parallelism: the
// chunks of each system are first split into G contiguous groups summed in
// order into tmp[s][g][e], then the G group sums are added in order.
template <typename ACC>
__global__ void reduce_groups_kernel(const ACC* __restrict__ partial,
                                     const int32_t* __restrict__ sys_begin, int64_t elems,
                                     int G, ACC* __restrict__ tmp) {
  const int s = blockIdx.y, g = blockIdx.z;
  const int c0 = sys_begin[s], c1 = sys_begin[s + 1];
  const int per = (c1 - c0 + G - 1) / G;
  const int a = min(c1, c0 + g * per), b = min(c1, a + per);
  ACC* t = tmp + ((int64_t)s * G + g) * elems;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    ACC v = 0;
    for (int c = a; c < b; ++c) v += partial[(int64_t)c * elems + e];
    t[e] = v;
  }
}
// The same over FP32 partials, four elements per thread, four chunks' loads in
// flight (same order of additions).
__global__ void reduce_groups4_kernel(const float* __restrict__ partial,
                                      const int32_t* __restrict__ sys_begin, int64_t elems, int G,
                                      float* __restrict__ tmp) {
  const int s = blockIdx.y, g = blockIdx.z;
  const int c0 = sys_begin[s], c1 = sys_begin[s + 1];
  const int per = (c1 - c0 + G - 1) / G;
  const int a = min(c1, c0 + g * per), b = min(c1, a + per);
  const int64_t n4 = elems >> 2;
  const float4* p4 = reinterpret_cast<const float4*>(partial);
  float4* t4 = reinterpret_cast<float4*>(tmp + ((int64_t)s * G + g) * elems);
  for (int64_t e4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e4 < n4;
       e4 += (int64_t)gridDim.x * blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    int c = a;
    for (; c + 4 <= b; c += 4) {
      float4 x[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) x[h] = __ldg(p4 + (int64_t)(c + h) * n4 + e4);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        v.x += x[h].x;
        v.y += x[h].y;
        v.z += x[h].z;
        v.w += x[h].w;
      }
    }
    for (; c < b; ++c) {
      const float4 x = __ldg(p4 + (int64_t)c * n4 + e4);
      v.x += x.x;
      v.y += x.y;
      v.z += x.z;
      v.w += x.w;
    }
    t4[e4] = v;
  }
}

template <typename ACC, typename OUT>
__global__ void reduce_group_sums_kernel(const ACC* __restrict__ tmp, int G, int64_t elems,
                                         OUT* __restrict__ out, int64_t out_sys_stride,
                                         int64_t seg, int64_t seg_stride, int accumulate) {
  const int s = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    OUT v = 0;
    for (int g = 0; g < G; ++g) v += (OUT)tmp[((int64_t)s * G + g) * elems + e];
    const int64_t h = e / seg;
    OUT* o = out + h * seg_stride + (int64_t)s * out_sys_stride + (e - h * seg);
    *o = accumulate ? *o + v : v;
  }
}

// Vector loads of CPT consecutive entries of a state row (CPT * element size
// is 4, 8, 16 or 32 bytes and the address is aligned to it).
template <int BYTES>
__device__ __forceinline__ void ld_words(const void* p, uint32_t* w) {
  if constexpr (BYTES == 4) {
    w[0] = *static_cast<const uint32_t*>(p);
  } else if constexpr (BYTES == 8) {
    const uint2 v = *static_cast<const uint2*>(p);
    w[0] = v.x; w[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < BYTES / 16; ++i) {
      const uint4 v = static_cast<const uint4*>(p)[i];
      w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
  }
}
template <int FMT, int CPT>
__device__ __forceinline__ void load_row_vec(const void* hi, const void* lo, int64_t idx,
                                             float* out) {
  if constexpr (FMT == FMT_BF16) {
    uint32_t h[CPT / 2], l[CPT / 2];
    ld_words<CPT * 2>(static_cast<const __nv_bfloat16*>(hi) + idx, h);
    ld_words<CPT * 2>(static_cast<const __nv_bfloat16*>(lo) + idx, l);
#pragma unroll
    for (int i = 0; i < CPT / 2; ++i) {
      // a BF16 value is the top half of the FP32 with the same bits
      out[2 * i] = __uint_as_float(h[i] << 16) + __uint_as_float(l[i] << 16);
      out[2 * i + 1] = __uint_as_float(h[i] & 0xffff0000u) + __uint_as_float(l[i] & 0xffff0000u);
    }
  } else {
    uint32_t h[CPT], l[CPT];
    ld_words<CPT * 4>(static_cast<const float*>(hi) + idx, h);
    ld_words<CPT * 4>(static_cast<const float*>(lo) + idx, l);
#pragma unroll
    for (int i = 0; i < CPT; ++i) out[i] = __uint_as_float(h[i]) + __uint_as_float(l[i]);
  }
}

// Wide-by-thin time reduction, for the products whose one side is narrow
// (p or q columns): for h < nsh and every row l of the chunk's tiles,
//   partial[chunk][h] += X_l (outer) T_(l - sh_h),
// X a state buffer or dense array with `a` columns, T dense [rows, ld] with tc
// columns (zero before the sequence start).  Each (chunk, h) block is stored
// [tc][a] if thin_major, else [a][tc].  A thread owns CPT consecutive columns
// of X (16-byte loads) and TT of the tt = nsh * tc thin columns: G column groups
// x TG thin groups of threads share a row, 256 / (G TG) rows are processed at
// once, and the row groups are summed in a fixed order, so the result is
// deterministic.
constexpr int WT_SMEM_BYTES = 32768;
constexpr int WT_TC_MAX = 16;   // thin columns per source (the rows staged in shared memory)
template <int FMT, typename ACC, int CPT, int TT>
__global__ void __launch_bounds__(256) wtreduce_kernel(const Tile* __restrict__ tiles,
                                                       const int32_t* __restrict__ chunks, int BM,
                                                       int m, TSrc X, int a,
                                                       const ACC* __restrict__ T, int ld, int tc,
                                                       int nsh, int sh0, int sh1, int gshift,
                                                       int tgshift, int vec, int thin_major,
                                                       ACC* __restrict__ partial) {
  __shared__ __align__(16) unsigned char red_raw[WT_SMEM_BYTES];
  // the tile's thin rows, times t0 - 1 .. t0 + BM - 1 (shifts are 0 or 1)
  constexpr int TROWS = (FMT == FMT_F64 ? 64 : 128) + 1;
  __shared__ ACC Ts[TROWS * WT_TC_MAX];
  ACC* red = reinterpret_cast<ACC*>(red_raw);
  const int c = blockIdx.x;
  const int first = chunks[3 * c], count = chunks[3 * c + 1];
  const int G = 1 << gshift, R = 256 >> (gshift + tgshift);
  const int g = threadIdx.x & (G - 1);
  const int tg = (threadIdx.x >> gshift) & ((1 << tgshift) - 1);
  const int rg = threadIdx.x >> (gshift + tgshift);
  const int i0 = g * CPT;
  const int e0 = tg * TT;           // this thread's first thin column
  const int tt = nsh * tc;
  ACC acc[CPT][TT];
#pragma unroll
  for (int i = 0; i < CPT; ++i)
#pragma unroll
    for (int e = 0; e < TT; ++e) acc[i][e] = 0;
  // rows in flight per thread: RU rows of CPT columns (32 values) are loaded
  // before their products; the thin values are read from shared memory
  constexpr int RU = 32 / CPT;
  for (int ti = first; ti < first + count; ++ti) {
    const Tile t = tiles[ti];
    const int rows = min(BM, t.len - t.t0);
    const int b = X.buf_mode ? t.fbuf : X.buf_fixed;
    __syncthreads();   // the previous tile's thin rows are no longer read
    for (int e = threadIdx.x; e < (rows + 1) * tc; e += 256) {
      const int r = e / tc, j = e - r * tc;
      const int l = t.t0 - 1 + r;
      Ts[r * WT_TC_MAX + j] = l >= 0 ? T[(t.seq_row0 + l) * ld + j] : (ACC)0;
    }
    __syncthreads();
    for (int rr0 = rg; rr0 < rows; rr0 += RU * R) {
      ACC xv[RU][CPT];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int rr = rr0 + u * R;
        const bool live = rr < rows && i0 < a;
        const int64_t row = t.seq_row0 + t.t0 + rr;
        if constexpr (FMT != FMT_F64) {
          if (vec && live) {
            float f[CPT];
            load_row_vec<FMT, CPT>(X.bufs.hi(b), X.bufs.lo(b), row * m + i0, f);
#pragma unroll
            for (int i = 0; i < CPT; ++i) xv[u][i] = f[i];
            continue;
          }
        }
#pragma unroll
        for (int i = 0; i < CPT; ++i)
          xv[u][i] = (live && i0 + i < a) ? (ACC)src_get<FMT>(X, t, row, i0 + i, m) : (ACC)0;
      }
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int rr = rr0 + u * R;
        if (rr >= rows) break;
        const int l = t.t0 + rr;
#pragma unroll
        for (int e = 0; e < TT; ++e) {
          const int eg = e0 + e;
          if (eg >= tt) break;
          const int h = eg >= tc ? 1 : 0;
          const int j = eg - h * tc;
          const int sh = h ? sh1 : sh0;
          const ACC tv = l - sh >= 0 ? Ts[(rr + 1 - sh) * WT_TC_MAX + j] : (ACC)0;
#pragma unroll
          for (int i = 0; i < CPT; ++i) acc[i][e] = fma(xv[u][i], tv, acc[i][e]);
        }
      }
    }
  }
  // Sum the row groups.  Single precision: every group stores its partial and
  // a pairwise tree with a fixed pairing adds them (log2 R barriers).  Double
  // precision (shared memory holds one partial): in group order.
  if constexpr (sizeof(ACC) == 4) {
    const int slab = a * tt;    // R * slab <= 256 * CPT * TT floats, within the buffer
    if (i0 < a) {
#pragma unroll
      for (int i = 0; i < CPT; ++i) {
        if (i0 + i >= a) continue;
#pragma unroll
        for (int e = 0; e < TT; ++e)
          if (e0 + e < tt) red[(int64_t)rg * slab + (i0 + i) * tt + e0 + e] = acc[i][e];
      }
    }
    for (int sstep = R >> 1; sstep >= 1; sstep >>= 1) {
      __syncthreads();
      if (rg < sstep && i0 < a) {
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
          if (i0 + i >= a) continue;
#pragma unroll
          for (int e = 0; e < TT; ++e)
            if (e0 + e < tt) {
              ACC* r0 = red + (int64_t)rg * slab + (i0 + i) * tt + e0 + e;
              *r0 += r0[(int64_t)sstep * slab];
            }
        }
      }
    }
    __syncthreads();
  } else {
    for (int q = 0; q < R; ++q) {
      if (rg == q) {
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
          if (i0 + i >= a) continue;
#pragma unroll
          for (int e = 0; e < TT; ++e) {
            if (e0 + e >= tt) continue;
            ACC* r = red + (int64_t)(i0 + i) * tt + e0 + e;
            *r = (q == 0 ? (ACC)0 : *r) + acc[i][e];
          }
        }
      }
      __syncthreads();
    }
  }
  const int64_t elems = (int64_t)a * tt;
  ACC* out = partial + (int64_t)c * elems;
  for (int64_t idx = threadIdx.x; idx < elems; idx += 256) {
    // idx in the output layout: [h][tc][a] or [h][a][tc]
    const int h = (int)(idx / ((int64_t)a * tc));
    const int rem = (int)(idx - (int64_t)h * a * tc);
    int i, j;
    if (thin_major) { j = rem / a; i = rem - j * a; }
    else { i = rem / tc; j = rem - i * tc; }
    out[idx] = red[(int64_t)i * tt + h * tc + j];
  }
}

// W^(N+1)_l = C^T G_l into adjoint buffer (N_i + 1) & 1 (tile.flags = N_i); thread per
// (row, column).
template <int FMT, typename T>
__global__ void __launch_bounds__(256) adj_init_kernel(const Tile* __restrict__ tiles, int BM,
                                                       int m, int q, const T* __restrict__ G,
                                                       const T* __restrict__ C, Bufs W) {
  const Tile t = tiles[blockIdx.x];
  const int rows = min(BM, t.len - t.t0);
  const int b = (t.flags + 1) & 1;
  void* hi = W.hi(b);
  void* lo = W.lo(b);
  const T* Cs = C + (int64_t)t.sys * q * m;
  for (int idx = threadIdx.x; idx < rows * m; idx += blockDim.x) {
    const int r = idx / m, col = idx % m;
    const int64_t row = t.seq_row0 + t.t0 + r;
    T acc = 0;
    for (int j = 0; j < q; ++j) acc = fma(Cs[(int64_t)j * m + col], G[row * q + j], acc);
    Store<FMT>::put(hi, lo, row * m + col, (double)acc);
  }
}

// du_l = Bbar^T W_l + (Abar Bbar)^T W_(l+1) + D^T G_l; one warp per row.
template <int FMT, typename T>
__global__ void __launch_bounds__(256) stage0_adj_kernel(const Tile* __restrict__ tiles, int BM,
                                                         int m, int p, int q,
                                                         const T* __restrict__ G,
                                                         const T* __restrict__ Bbar,
                                                         const T* __restrict__ ABbar,
                                                         const T* __restrict__ D, Bufs W, int wbuf,
                                                         T* __restrict__ du) {
  const Tile t = tiles[blockIdx.x];
  const int rows = min(BM, t.len - t.t0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const void* wh = W.hi(wbuf);
  const void* wl = W.lo(wbuf);
  const T* Bs = Bbar + (int64_t)t.sys * m * p;
  const T* ABs = ABbar + (int64_t)t.sys * m * p;
  const T* Ds = D + (int64_t)t.sys * q * p;
  for (int r = warp; r < rows; r += nw) {
    const int l = t.t0 + r;
    const int64_t row = t.seq_row0 + l;
    const bool next = l + 1 < t.len;
    for (int j = 0; j < p; ++j) {
      T s = 0;
      for (int c = lane; c < m; c += 32) {
        s = fma(Bs[(int64_t)c * p + j], (T)load_elem<FMT>(wh, wl, row * m + c), s);
        if (next) s = fma(ABs[(int64_t)c * p + j], (T)load_elem<FMT>(wh, wl, (row + 1) * m + c), s);
      }
      for (int c = lane; c < q; c += 32) s = fma(Ds[(int64_t)c * p + j], G[row * q + c], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) du[row * p + j] = (T)s;
    }
  }
}

// Batched transpose: out[b][j][i] = in[b][i][j] for n x n matrices.
__global__ void transpose_kernel(const double* __restrict__ in, double* __restrict__ out, int n,
                                 int64_t stride) {
  __shared__ double tile[32][33];
  const double* src = in + (int64_t)blockIdx.z * stride;
  double* dst = out + (int64_t)blockIdx.z * stride;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int i = y0 + yy, j = x0 + threadIdx.x;
    if (i < n && j < n) tile[yy][threadIdx.x] = src[(int64_t)i * n + j];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int j = x0 + yy, i = y0 + threadIdx.x;
    if (i < n && j < n) dst[(int64_t)j * n + i] = tile[threadIdx.x][yy];
  }
}

// y[s][e] = (accumulate ? y[s][e] : 0) + factor * scal[s] * x[s][e]   (scal may be null: 1)
template <typename T>
__global__ void axpy_sys_kernel(const T* __restrict__ x, int64_t x_stride, T* __restrict__ y,
                                int64_t y_stride, int64_t n, const double* __restrict__ scal,
                                double factor, int accumulate) {
  const int s = blockIdx.y;
  const T a = (T)(factor * (scal ? scal[s] : 1.0));
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T v = a * x[(int64_t)s * x_stride + e];
    T* o = y + (int64_t)s * y_stride + e;
    *o = accumulate ? *o + v : v;
  }
}

// out[s][i] = (T_out) in[s][i] over strided batches (precision conversion).
template <typename TI, typename TO>
__global__ void convert_sys_kernel(const TI* __restrict__ in, int64_t in_stride,
                                   TO* __restrict__ out, int64_t out_stride, int64_t n) {
  const int s = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)s * out_stride + e] = (TO)in[(int64_t)s * in_stride + e];
}

}  // namespace

// First-stage adjoint for narrow p and q, one pass over W = W^(1):
//   du_l = Bbar^T W_l + (Abar Bbar)^T W_(l+1) + D^T G_l        (W past the sequence end is 0)
//   R1  += W_l u_l^T,   R2 += W_l u_(l-1)^T                     (u before the start is 0)
// One block per chunk of tiles (one system), eight warps.  A warp walks 16 rows of
// each tile plus the next row (whose (Abar Bbar)^T W completes the warp's last du);
// lane l owns the 8-column groups 8 (l + 32 g), g < NG, of every row, so a row is one
// coalesced read and the two p-wide dot products of du are warp reductions.  The
// rows are read in batches of RB; each thread copies its own 16-byte pieces of the
// batch FA_ST - 1 ahead into shared memory (cp.async), and the first lanes of a warp
// copy the batch's u and G values, so the loads stay in flight while earlier rows
// are reduced.  The warps' R1, R2 partials are added in a fixed order into
// partial[chunk][h][i][j] (h = 0: R1, 1: R2), summed per system afterwards.
constexpr int FA_PMAX = 4;   // p, q <= 4
constexpr int FA_CMAX = 2;   // NG * p <= 2 (accumulators per lane: 2 x 8 x NG x p)
constexpr int FA_ST = 3;     // batches in shared memory (FA_ST - 1 in flight)
constexpr int FA_SW = 8;     // 16-byte words a thread copies per batch
template <int FMT>
__host__ __device__ constexpr int fa_vw() { return FMT == FMT_BF16 ? 1 : 2; }   // words / 8 cols
template <int FMT, int CM>
__host__ __device__ constexpr int fa_rb() { return FA_SW / (CM * 2 * fa_vw<FMT>()); }
__host__ __device__ constexpr int fa_scalars(int rb, int pm) { return rb * 3 * pm; }
// Shared memory: the batch ring, then the scalar ring; the R1, R2 reduction
// at the end reuses the space.
__host__ __device__ constexpr size_t fa_smem_bytes(int rb, int pm) {
  return (size_t)FA_ST * FA_SW * 256 * 16 + (size_t)FA_ST * 8 * fa_scalars(rb, pm) * 4;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(ptx::smem_addr(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(ptx::smem_addr(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// CM >= NG * p: accumulator groups per lane; PM >= p, q
template <int FMT, int CM, int PM>
__global__ void __launch_bounds__(256, 2) first_adj_thin_kernel(
    const Tile* __restrict__ tiles, const int32_t* __restrict__ chunks, int m, int p, int q,
    Bufs W, int wbuf, const float* __restrict__ u, const float* __restrict__ G,
    const float* __restrict__ Bbar, const float* __restrict__ ABbar,
    const float* __restrict__ D, float* __restrict__ du, float* __restrict__ partial) {
  extern __shared__ __align__(16) float fa_smem[];
  constexpr int VW = fa_vw<FMT>();
  constexpr int RB = fa_rb<FMT, CM>();      // rows per batch
  constexpr int NBT = 16 / RB + 1;          // batches per tile: rows r0 .. r0 + 16
  constexpr int SC = fa_scalars(RB, PM);    // u_l, u_(l-1), G_(l-1) of a batch
  constexpr int ELEM = FMT == FMT_BF16 ? 2 : 4;
  static_assert(RB >= 1 && RB * CM * 2 * VW == FA_SW, "batch words");
  uint4* ring = reinterpret_cast<uint4*>(fa_smem);                   // [FA_ST][FA_SW][256]
  float* scal = reinterpret_cast<float*>(ring + FA_ST * FA_SW * 256);   // [FA_ST][8][SC]
  const int c = blockIdx.x;
  const int first = chunks[3 * c], count = chunks[3 * c + 1], sys = chunks[3 * c + 2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NG = (m + 255) / 256;
  const char* wh = static_cast<const char*>(W.hi(wbuf));
  const char* wl = static_cast<const char*>(W.lo(wbuf));
  // this lane's coefficients: Bbar[col][j], ABbar[col][j]
  float cb[CM][8], cab[CM][8];
  float acc1[CM][8], acc2[CM][8];
#pragma unroll
  for (int gj = 0; gj < CM; ++gj) {
    const int g = gj / p, j = gj - g * p;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = 8 * (lane + 32 * g) + e;
      const bool ok = gj < NG * p && col < m;
      cb[gj][e] = ok ? Bbar[((int64_t)sys * m + col) * p + j] : 0.f;
      cab[gj][e] = ok ? ABbar[((int64_t)sys * m + col) * p + j] : 0.f;
      acc1[gj][e] = 0.f;
      acc2[gj][e] = 0.f;
    }
  }
  float Ds[PM][PM];
#pragma unroll
  for (int i = 0; i < PM; ++i)
#pragma unroll
    for (int j = 0; j < PM; ++j)
      Ds[i][j] = (i < q && j < p) ? D[((int64_t)sys * q + i) * p + j] : 0.f;

  const int r0 = 16 * warp;
  const int nb = count * NBT;
  // Batch b: rows r0 + (b % NBT) RB .. + RB - 1 of tile first + b / NBT.  Every
  // call commits one group (empty past the end), so wait_group counts batches.
  auto issue = [&](int b) {
    if (b < nb) {
      const Tile t = tiles[first + b / NBT];
      const int rb = r0 + (b % NBT) * RB;
      const int st = b % FA_ST;
#pragma unroll
      for (int v = 0; v < RB; ++v) {
        const int l = t.t0 + rb + v;
        const bool live = rb + v <= r0 + 16 && l < t.len;
        const int64_t row = t.seq_row0 + l;
#pragma unroll
        for (int g = 0; g < CM; ++g) {
          const int col0 = 8 * (lane + 32 * g);
          const bool ok = live && g < NG && col0 < m;
          const int64_t off = ok ? (row * m + col0) * ELEM : 0;
#pragma unroll
          for (int w = 0; w < VW; ++w) {
            uint4* dh = ring + ((st * FA_SW) + ((v * CM + g) * 2 + 0) * VW + w) * 256 + threadIdx.x;
            uint4* dl = ring + ((st * FA_SW) + ((v * CM + g) * 2 + 1) * VW + w) * 256 + threadIdx.x;
            cp_async16(dh, wh + off + 16 * w, ok ? 16 : 0);
            cp_async16(dl, wl + off + 16 * w, ok ? 16 : 0);
          }
        }
      }
      for (int e = lane; e < SC; e += 32) {
        const int v = e / (3 * PM), kind = (e / PM) % 3, j = e % PM;
        const int l = t.t0 + rb + v;
        const int64_t row = t.seq_row0 + l;
        const bool in16 = rb + v <= r0 + 16;
        bool ok;
        const float* src;
        if (kind == 0) {
          ok = in16 && l < t.len && j < p;
          src = u + row * p + j;
        } else if (kind == 1) {
          ok = in16 && l < t.len && j < p && l >= 1;
          src = u + (row - 1) * p + j;
        } else {
          ok = in16 && l >= 1 && l - 1 < t.len && j < q;
          src = G + (row - 1) * q + j;
        }
        cp_async4(scal + (st * 8 + warp) * SC + e, ok ? src : u, ok ? 4 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int b = 0; b < FA_ST - 1; ++b) issue(b);

  float aprev[PM];
  for (int b = 0; b < nb; ++b) {
    issue(b + FA_ST - 1);
    cp_async_wait<FA_ST - 1>();   // this thread's copies of batch b have landed
    __syncwarp();                 // and the other lanes' scalar copies
    const Tile t = tiles[first + b / NBT];
    const int rb = r0 + (b % NBT) * RB;
    const int st = b % FA_ST;
    if (rb == r0) {
#pragma unroll
      for (int j = 0; j < PM; ++j) aprev[j] = 0.f;
    }
    const float* sb = scal + (st * 8 + warp) * SC;
#pragma unroll
    for (int v = 0; v < RB; ++v) {
      const int r = rb + v;
      if (r > r0 + 16) break;
      float xs[CM][8];
#pragma unroll
      for (int g = 0; g < CM; ++g) {
        const uint4* sh = ring + ((st * FA_SW) + ((v * CM + g) * 2 + 0) * VW) * 256 + threadIdx.x;
        const uint4* sl = ring + ((st * FA_SW) + ((v * CM + g) * 2 + 1) * VW) * 256 + threadIdx.x;
        if constexpr (FMT == FMT_BF16) {
          const uint4 h4 = sh[0], l4 = sl[0];
          const uint32_t h[4] = {h4.x, h4.y, h4.z, h4.w}, lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            // a BF16 value is the top half of the FP32 with the same bits
            xs[g][2 * i] = __uint_as_float(h[i] << 16) + __uint_as_float(lw[i] << 16);
            xs[g][2 * i + 1] =
                __uint_as_float(h[i] & 0xffff0000u) + __uint_as_float(lw[i] & 0xffff0000u);
          }
        } else {
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const uint4 h4 = sh[w * 256], l4 = sl[w * 256];
            xs[g][4 * w + 0] = __uint_as_float(h4.x) + __uint_as_float(l4.x);
            xs[g][4 * w + 1] = __uint_as_float(h4.y) + __uint_as_float(l4.y);
            xs[g][4 * w + 2] = __uint_as_float(h4.z) + __uint_as_float(l4.z);
            xs[g][4 * w + 3] = __uint_as_float(h4.w) + __uint_as_float(l4.w);
          }
        }
      }
      const int l = t.t0 + r;                 // time step in the sequence
      const bool live = l < t.len;
      const int64_t row = t.seq_row0 + l;
      // lane partials of Bbar^T W_l and (Abar Bbar)^T W_l, then warp sums
      float a[PM], bsum[PM];
#pragma unroll
      for (int j = 0; j < PM; ++j) { a[j] = 0.f; bsum[j] = 0.f; }
#pragma unroll
      for (int gj = 0; gj < CM; ++gj) {
        if (gj >= NG * p) break;
        const int g = gj / p, j = gj - g * p;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          a[j] = fmaf(cb[gj][e], xs[g][e], a[j]);
          bsum[j] = fmaf(cab[gj][e], xs[g][e], bsum[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < PM; ++j) {
        if (j >= p) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a[j] += __shfl_xor_sync(0xffffffffu, a[j], o);
          bsum[j] += __shfl_xor_sync(0xffffffffu, bsum[j], o);
        }
      }
      // du of the previous row: Bbar^T W_(l-1) + (Abar Bbar)^T W_l + D^T G_(l-1)
      if (r > r0 && lane == 0 && l - 1 < t.len) {
        const int64_t prow = row - 1;
#pragma unroll
        for (int j = 0; j < PM; ++j) {
          if (j >= p) break;
          float val = aprev[j] + bsum[j];
#pragma unroll
          for (int i = 0; i < PM; ++i) val = fmaf(Ds[i][j], sb[v * 3 * PM + 2 * PM + i], val);
          du[prow * p + j] = val;
        }
      }
#pragma unroll
      for (int j = 0; j < PM; ++j) aprev[j] = a[j];
      // R1 += W_l u_l^T, R2 += W_l u_(l-1)^T over the warp's own rows
      if (r < r0 + 16 && live) {
#pragma unroll
        for (int gj = 0; gj < CM; ++gj) {
          if (gj >= NG * p) break;
          const int g = gj / p, j = gj - g * p;
          const float u1 = sb[v * 3 * PM + j], u0 = sb[v * 3 * PM + PM + j];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            acc1[gj][e] = fmaf(xs[g][e], u1, acc1[gj][e]);
            acc2[gj][e] = fmaf(xs[g][e], u0, acc2[gj][e]);
          }
        }
      }
    }
    __syncwarp();   // every lane has read the scalars of slot st before it is refilled
  }
  cp_async_wait<0>();
  __syncthreads();   // the ring is reused for the reduction below
  // the warps' partials, added in warp order
  float* fa_red = fa_smem;   // [8 warps][2][m][p]
  const int mp = m * p;
#pragma unroll
  for (int gj = 0; gj < CM; ++gj) {
    if (gj >= NG * p) break;
    const int g = gj / p, j = gj - g * p;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = 8 * (lane + 32 * g) + e;
      if (col < m) {
        fa_red[(warp * 2 + 0) * mp + col * p + j] = acc1[gj][e];
        fa_red[(warp * 2 + 1) * mp + col * p + j] = acc2[gj][e];
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * mp; e += blockDim.x) {
    const int h = e / mp, idx = e - h * mp;
    float v = 0.f;
    for (int w8 = 0; w8 < 8; ++w8) v += fa_red[(w8 * 2 + h) * mp + idx];
    partial[(int64_t)c * 2 * mp + e] = v;
  }
}

bool first_adj_thin_supported(const Plan& p) {
  const int NG = (p.d.m + 255) / 256;
  return p.d.precision != CASCADE_FP64 && tile_rows(p) == 128 && p.d.m % 8 == 0 &&
         p.d.p <= FA_PMAX && p.d.q <= FA_PMAX && NG * p.d.p <= FA_CMAX;
}

// ------------------------------------------------------------------ launchers
// Sum the chunk partials of every system into out (see reduce_partials_kernel),
// in two grouped passes when systems x elements alone cannot fill the GPU.
template <typename ACC, typename OUT>
static void sum_chunks(const Plan& p, const ACC* partial, const int32_t* sys_begin,
                       int64_t elems, OUT* out, int64_t out_sys_stride, int64_t seg,
                       int64_t seg_stride, int accumulate, cudaStream_t st) {
  const int rblocks = (int)((elems + 255) / 256 < 1024 ? (elems + 255) / 256 : 1024);
  // threads that keep the GPU busy; the FP32 kernels take four elements each
  const bool vec = sizeof(ACC) == 4 && elems % 4 == 0;
  const int64_t want = (int64_t)2048 * p.num_sms;
  const int64_t have = elems * p.d.nsys / (vec ? 4 : 1);
  int G = 1;
  if (have < want && p.d_red_scratch) {
    G = (int)std::min<int64_t>(32, (want + have - 1) / have);
    while (G > 1 && (size_t)G * elems * p.d.nsys * sizeof(ACC) > p.red_scratch_bytes) --G;
    if (G < 3) G = 1;   // two passes pay off only for a few groups or more
  }
  if (G <= 1) {
    if (sizeof(ACC) == 4 && elems % 4 == 0 &&
        reinterpret_cast<uintptr_t>(partial) % 16 == 0) {
      const int64_t n4 = elems / 4;
      const int b4 = (int)std::min<int64_t>((n4 + 255) / 256, 4 * (int64_t)p.num_sms);
      reduce_partials4_kernel<OUT><<<dim3(b4, p.d.nsys), 256, 0, st>>>(
          reinterpret_cast<const float*>(partial), sys_begin, elems, out, out_sys_stride, seg,
          seg_stride, accumulate);
      CASCADE_LAUNCHED();
      return;
    }
    reduce_partials_kernel<ACC, OUT><<<dim3(rblocks, p.d.nsys), 256, 0, st>>>(
        partial, sys_begin, elems, out, out_sys_stride, seg, seg_stride, accumulate);
    CASCADE_LAUNCHED();
    return;
  }
  ACC* tmp = static_cast<ACC*>(p.d_red_scratch);
  if (sizeof(ACC) == 4 && elems % 4 == 0 && reinterpret_cast<uintptr_t>(partial) % 16 == 0 &&
      reinterpret_cast<uintptr_t>(tmp) % 16 == 0) {
    const int b4 = (int)std::min<int64_t>((elems / 4 + 255) / 256, 1024);
    reduce_groups4_kernel<<<dim3(b4, p.d.nsys, G), 256, 0, st>>>(
        reinterpret_cast<const float*>(partial), sys_begin, elems, G,
        reinterpret_cast<float*>(tmp));
  } else {
    reduce_groups_kernel<ACC><<<dim3(rblocks, p.d.nsys, G), 256, 0, st>>>(partial, sys_begin,
                                                                          elems, G, tmp);
  }
  CASCADE_LAUNCHED();
  reduce_group_sums_kernel<ACC, OUT><<<dim3(rblocks, p.d.nsys), 256, 0, st>>>(
      tmp, G, elems, out, out_sys_stride, seg, seg_stride, accumulate);
  CASCADE_LAUNCHED();
}

cudaError_t launch_treduce(const Plan& p, const Tile* tiles, const int32_t* chunks, int nchunks,
                           const int32_t* sys_begin, const TSrc& X, int a, const TSrc& Y, int b,
                           int shift, void* partial, void* out, bool out_f64,
                           int64_t out_sys_stride, int accumulate, cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  const int BM = tile_rows(p);
  const TSrc xs = X, ys = Y;
  dim3 grid((b + 63) / 64, (a + 63) / 64, nchunks);
  const int64_t elems = (int64_t)a * b;
  if (p.d.precision == CASCADE_FP64) {
    treduce_kernel<FMT_F64, double><<<grid, 256, 0, st>>>(tiles, chunks, BM, p.d.m, xs, a, ys, b,
                                                         shift, (double*)partial);
    CASCADE_LAUNCHED();
    sum_chunks<double, double>(p, (const double*)partial, sys_begin, elems, (double*)out,
                               out_sys_stride, elems, 0, accumulate, st);
  } else {
    if (p.d.precision == CASCADE_BF16_SPLIT)
      treduce_kernel<FMT_BF16, float><<<grid, 256, 0, st>>>(tiles, chunks, BM, p.d.m, xs, a, ys, b,
                                                           shift, (float*)partial);
    else
      treduce_kernel<FMT_F32, float><<<grid, 256, 0, st>>>(tiles, chunks, BM, p.d.m, xs, a, ys, b,
                                                          shift, (float*)partial);
    CASCADE_LAUNCHED();
    if (out_f64)
      sum_chunks<float, double>(p, (const float*)partial, sys_begin, elems, (double*)out,
                                out_sys_stride, elems, 0, accumulate, st);
    else
      sum_chunks<float, float>(p, (const float*)partial, sys_begin, elems, (float*)out,
                               out_sys_stride, elems, 0, accumulate, st);
  }
  return cudaGetLastError();
}

// Thread shape of the wide-by-thin reduction: CPT columns per thread for TT
// thin columns (CPT * TT <= 32 accumulators).
// Thread shape of the wide-by-thin reduction: 8 columns per thread, TT thin
// columns per thread (at most 4, so 32 accumulators), TG thin groups per row.
static int wt_tt(int tt) { return tt <= 1 ? 1 : tt <= 2 ? 2 : 4; }
static int wt_tg(int tt) {
  const int TT = wt_tt(tt);
  int tg = 1;
  while (tg * TT < tt) tg <<= 1;
  return tg;
}

bool wtreduce_supported(const Plan& p, int a, int tc, int nsh) {
  const int tt = nsh * tc;
  if (nsh < 1 || nsh > 2 || tc < 1 || tc > WT_TC_MAX || tt > 32) return false;
  int G = 1;
  while (G * 8 < a) G <<= 1;
  if (G * wt_tg(tt) > 256) return false;
  const size_t acc = p.d.precision == CASCADE_FP64 ? 8 : 4;
  return (size_t)a * tt * acc <= (size_t)WT_SMEM_BYTES;
}

template <int FMT, typename ACC, int CPT, int TT>
static void wt_launch(int nchunks, const Tile* tiles, const int32_t* chunks, int BM, int m,
                      const TSrc& X, int a, const ACC* T, int ld, int tc, int nsh, int sh0,
                      int sh1, int gshift, int tgshift, int vec, int thin_major, ACC* partial,
                      cudaStream_t st) {
  wtreduce_kernel<FMT, ACC, CPT, TT><<<nchunks, 256, 0, st>>>(tiles, chunks, BM, m, X, a, T, ld,
                                                              tc, nsh, sh0, sh1, gshift, tgshift,
                                                              vec, thin_major, partial);
}

template <int FMT, typename ACC>
static void wt_dispatch(int TT, int nchunks, const Tile* tiles, const int32_t* chunks, int BM,
                        int m, const TSrc& X, int a, const ACC* T, int ld, int tc, int nsh,
                        int sh0, int sh1, int gshift, int tgshift, int vec, int thin_major,
                        ACC* partial, cudaStream_t st) {
  if (TT == 1)
    wt_launch<FMT, ACC, 8, 1>(nchunks, tiles, chunks, BM, m, X, a, T, ld, tc, nsh, sh0, sh1,
                              gshift, tgshift, vec, thin_major, partial, st);
  else if (TT == 2)
    wt_launch<FMT, ACC, 8, 2>(nchunks, tiles, chunks, BM, m, X, a, T, ld, tc, nsh, sh0, sh1,
                              gshift, tgshift, vec, thin_major, partial, st);
  else
    wt_launch<FMT, ACC, 8, 4>(nchunks, tiles, chunks, BM, m, X, a, T, ld, tc, nsh, sh0, sh1,
                              gshift, tgshift, vec, thin_major, partial, st);
}

cudaError_t launch_wtreduce(const Plan& p, const Tile* tiles, const int32_t* chunks, int nchunks,
                            const int32_t* sys_begin, const TSrc& X, int a, const void* T, int tc,
                            int nsh, int sh0, int sh1, bool thin_major, void* partial, void* out,
                            bool out_f64, int64_t out_sys_stride, int64_t seg_stride,
                            cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  if (!wtreduce_supported(p, a, tc, nsh) || sh0 < 0 || sh0 > 1 || sh1 < 0 || sh1 > 1)
    return cudaErrorInvalidValue;
  const int BM = tile_rows(p);
  const int TT = wt_tt(nsh * tc);
  const int CPT = 8;
  int gshift = 0, tgshift = 0;
  while ((1 << gshift) < (a + CPT - 1) / CPT) ++gshift;
  while ((1 << tgshift) < wt_tg(nsh * tc)) ++tgshift;
  // vector loads: a state buffer whose rows the column groups cover exactly
  const int vec = (X.kind == 0 && a == p.d.m && a % CPT == 0) ? 1 : 0;
  const int64_t elems = (int64_t)nsh * a * tc;
  const int64_t seg = (int64_t)a * tc;
  if (p.d.precision == CASCADE_FP64) {
    wt_dispatch<FMT_F64, double>(TT, nchunks, tiles, chunks, BM, p.d.m, X, a,
                                 static_cast<const double*>(T), tc, tc, nsh, sh0, sh1, gshift, tgshift, 0,
                                 thin_major ? 1 : 0, static_cast<double*>(partial), st);
    CASCADE_LAUNCHED();
    sum_chunks<double, double>(p, (const double*)partial, sys_begin, elems, (double*)out,
                               out_sys_stride, seg, seg_stride, 0, st);
  } else {
    if (p.d.precision == CASCADE_BF16_SPLIT)
      wt_dispatch<FMT_BF16, float>(TT, nchunks, tiles, chunks, BM, p.d.m, X, a,
                                   static_cast<const float*>(T), tc, tc, nsh, sh0, sh1, gshift, tgshift, vec,
                                   thin_major ? 1 : 0, static_cast<float*>(partial), st);
    else
      wt_dispatch<FMT_F32, float>(TT, nchunks, tiles, chunks, BM, p.d.m, X, a,
                                  static_cast<const float*>(T), tc, tc, nsh, sh0, sh1, gshift, tgshift, vec,
                                  thin_major ? 1 : 0, static_cast<float*>(partial), st);
    CASCADE_LAUNCHED();
    if (out_f64)
      sum_chunks<float, double>(p, (const float*)partial, sys_begin, elems, (double*)out,
                                out_sys_stride, seg, seg_stride, 0, st);
    else
      sum_chunks<float, float>(p, (const float*)partial, sys_begin, elems, (float*)out,
                               out_sys_stride, seg, seg_stride, 0, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const Plan& p, const float* partial, const int32_t* sys_begin,
                                   int64_t elems, void* out, bool out_f64, int64_t out_sys_stride,
                                   cudaStream_t st) {
  if (out_f64)
    sum_chunks<float, double>(p, partial, sys_begin, elems, (double*)out, out_sys_stride, elems,
                              0, 0, st);
  else
    sum_chunks<float, float>(p, partial, sys_begin, elems, (float*)out, out_sys_stride, elems, 0,
                             0, st);
  return cudaGetLastError();
}

// du (FP32 [rows, p]) and R1, R2 (out, out + seg_stride; [nsys, m, p] each) from W^(1)
// (buffer wbuf of W) in one pass; see first_adj_thin_kernel.
cudaError_t launch_first_adj_thin(const Plan& p, const Tile* tiles, const int32_t* chunks,
                                  int nchunks, const int32_t* sys_begin, const Bufs& W, int wbuf,
                                  const float* u, const float* G, float* du, float* partial,
                                  void* out, bool out_f64, int64_t out_sys_stride,
                                  int64_t seg_stride, cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  if (!first_adj_thin_supported(p)) return cudaErrorInvalidValue;
  const int m = p.d.m, pp = p.d.p, q = p.d.q;
  const int cm = ((m + 255) / 256) * pp;
  const bool bf = p.d.precision == CASCADE_BF16_SPLIT;
  const bool one = pp == 1 && q == 1;
  const int rb = cm <= 1 ? (bf ? fa_rb<FMT_BF16, 1>() : fa_rb<FMT_F32, 1>())
                         : (bf ? fa_rb<FMT_BF16, 2>() : fa_rb<FMT_F32, 2>());
  const size_t red = (size_t)8 * 2 * m * pp * sizeof(float);
  const size_t ring = fa_smem_bytes(rb, cm <= 1 && one ? 1 : FA_PMAX);
  const size_t smem = ring > red ? ring : red;
  auto kern = cm <= 1 ? (one ? (bf ? first_adj_thin_kernel<FMT_BF16, 1, 1>
                                   : first_adj_thin_kernel<FMT_F32, 1, 1>)
                             : (bf ? first_adj_thin_kernel<FMT_BF16, 1, FA_PMAX>
                                   : first_adj_thin_kernel<FMT_F32, 1, FA_PMAX>))
                      : (bf ? first_adj_thin_kernel<FMT_BF16, 2, FA_PMAX>
                            : first_adj_thin_kernel<FMT_F32, 2, FA_PMAX>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nchunks, 256, smem, st>>>(tiles, chunks, m, pp, q, W, wbuf, u, G, p.Bbar32, p.ABbar32,
                                   p.D32, du, partial);
  CASCADE_LAUNCHED();
  const int64_t elems = (int64_t)2 * m * pp, seg = (int64_t)m * pp;
  if (out_f64)
    sum_chunks<float, double>(p, partial, sys_begin, elems, (double*)out, out_sys_stride, seg,
                              seg_stride, 0, st);
  else
    sum_chunks<float, float>(p, partial, sys_begin, elems, (float*)out, out_sys_stride, seg,
                             seg_stride, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_adj_init(const Plan& p, const void* G, const Bufs& W, cudaStream_t st) {
  const int n = p.n_all_tiles;
  if (n == 0) return cudaSuccess;
  const int BM = tile_rows(p);
  switch (p.d.precision) {
    case CASCADE_FP64:
      adj_init_kernel<FMT_F64, double><<<n, 256, 0, st>>>(p.d_all_tiles, BM, p.d.m, p.d.q,
                                                          (const double*)G, p.C64, W);
      break;
    case CASCADE_BF16_SPLIT:
      adj_init_kernel<FMT_BF16, float><<<n, 256, 0, st>>>(p.d_all_tiles, BM, p.d.m, p.d.q,
                                                          (const float*)G, p.C32, W);
      break;
    default:
      adj_init_kernel<FMT_F32, float><<<n, 256, 0, st>>>(p.d_all_tiles, BM, p.d.m, p.d.q,
                                                         (const float*)G, p.C32, W);
  }
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_stage0_adj(const Plan& p, const void* G, const Bufs& W, int wbuf, void* du,
                              cudaStream_t st) {
  const int n = p.n_all_tiles;
  if (n == 0) return cudaSuccess;
  const int BM = tile_rows(p);
  switch (p.d.precision) {
    case CASCADE_FP64:
      stage0_adj_kernel<FMT_F64, double><<<n, 256, 0, st>>>(
          p.d_all_tiles, BM, p.d.m, p.d.p, p.d.q, (const double*)G, p.Bbar64, p.ABbar64, p.D64,
          W, wbuf, (double*)du);
      break;
    case CASCADE_BF16_SPLIT:
      stage0_adj_kernel<FMT_BF16, float><<<n, 256, 0, st>>>(
          p.d_all_tiles, BM, p.d.m, p.d.p, p.d.q, (const float*)G, p.Bbar32, p.ABbar32, p.D32, W,
          wbuf, (float*)du);
      break;
    default:
      stage0_adj_kernel<FMT_F32, float><<<n, 256, 0, st>>>(
          p.d_all_tiles, BM, p.d.m, p.d.p, p.d.q, (const float*)G, p.Bbar32, p.ABbar32, p.D32, W,
          wbuf, (float*)du);
  }
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_transpose(const double* in, double* out, int n, int64_t stride, int batch,
                             cudaStream_t st) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  dim3 grid((n + 31) / 32, (n + 31) / 32, batch);
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, out, n, stride);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy_sys(const T* x, int64_t x_stride, T* y, int64_t y_stride, int64_t n,
                            int nsys, const double* scal, double factor, bool accumulate,
                            cudaStream_t st) {
  if (n <= 0 || nsys <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  axpy_sys_kernel<T><<<dim3(blocks, nsys), 256, 0, st>>>(x, x_stride, y, y_stride, n, scal,
                                                         factor, accumulate ? 1 : 0);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}
template cudaError_t launch_axpy_sys<double>(const double*, int64_t, double*, int64_t, int64_t,
                                             int, const double*, double, bool, cudaStream_t);
template cudaError_t launch_axpy_sys<float>(const float*, int64_t, float*, int64_t, int64_t, int,
                                            const double*, double, bool, cudaStream_t);

template <typename TI, typename TO>
cudaError_t launch_convert_sys(const TI* in, int64_t in_stride, TO* out, int64_t out_stride,
                               int64_t n, int nsys, cudaStream_t st) {
  if (n <= 0 || nsys <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  convert_sys_kernel<TI, TO><<<dim3(blocks, nsys), 256, 0, st>>>(in, in_stride, out, out_stride, n);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}
template cudaError_t launch_convert_sys<double, float>(const double*, int64_t, float*, int64_t,
                                                       int64_t, int, cudaStream_t);
template cudaError_t launch_convert_sys<float, double>(const float*, int64_t, double*, int64_t,
                                                       int64_t, int, cudaStream_t);

}  // namespace cascade
