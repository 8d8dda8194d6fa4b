// formats.cuh -- element access to the state formats of the workspace.
//
// A state row of m entries is stored as one FP64 plane (FP64 plans), as a
// (hi, lo) pair of BF16 planes (hi = RN_bf16(x), lo = RN_bf16(x - hi)), or as
// a (hi, lo) pair of TF32-exact FP32 planes.  Dense inputs (u, dy) are plain
// FP32 or FP64 arrays.
#pragma once
#include "common.cuh"
#include "ptx.cuh"

namespace cascade {

enum { FMT_F64 = 0, FMT_BF16 = 2, FMT_F32 = 4 };

template <int FMT>
struct Store;
template <>
struct Store<FMT_F64> {
  static __device__ __forceinline__ void put(void* hi, void*, int64_t i, double v) {
    static_cast<double*>(hi)[i] = v;
  }
  static __device__ __forceinline__ double get(const void* hi, const void*, int64_t i) {
    return static_cast<const double*>(hi)[i];
  }
};
template <>
struct Store<FMT_BF16> {
  static __device__ __forceinline__ void put(void* hi, void* lo, int64_t i, double v) {
    const float x = (float)v;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    static_cast<__nv_bfloat16*>(hi)[i] = h;
    static_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
  static __device__ __forceinline__ double get(const void* hi, const void* lo, int64_t i) {
    return (double)(__bfloat162float(static_cast<const __nv_bfloat16*>(hi)[i]) +
                    __bfloat162float(static_cast<const __nv_bfloat16*>(lo)[i]));
  }
};
template <>
struct Store<FMT_F32> {
  static __device__ __forceinline__ void put(void* hi, void* lo, int64_t i, double v) {
    const float x = (float)v;
    const float h = ptx::tf32_rna(x);
    static_cast<float*>(hi)[i] = h;
    static_cast<float*>(lo)[i] = ptx::tf32_rna(x - h);
  }
  static __device__ __forceinline__ double get(const void* hi, const void* lo, int64_t i) {
    return (double)(static_cast<const float*>(hi)[i] + static_cast<const float*>(lo)[i]);
  }
};

// Element load in the arithmetic type of the format: double for the FP64
// plane, float for the tensor-core pairs (FP64 arithmetic is slow on GB300).
template <int FMT>
struct Acc {
  typedef float type;
};
template <>
struct Acc<FMT_F64> {
  typedef double type;
};
template <int FMT>
__device__ __forceinline__ typename Acc<FMT>::type load_elem(const void* hi, const void* lo,
                                                             int64_t i);
template <>
__device__ __forceinline__ double load_elem<FMT_F64>(const void* hi, const void*, int64_t i) {
  return static_cast<const double*>(hi)[i];
}
template <>
__device__ __forceinline__ float load_elem<FMT_BF16>(const void* hi, const void* lo, int64_t i) {
  return __bfloat162float(static_cast<const __nv_bfloat16*>(hi)[i]) +
         __bfloat162float(static_cast<const __nv_bfloat16*>(lo)[i]);
}
template <>
__device__ __forceinline__ float load_elem<FMT_F32>(const void* hi, const void* lo, int64_t i) {
  return static_cast<const float*>(hi)[i] + static_cast<const float*>(lo)[i];
}

}  // namespace cascade
