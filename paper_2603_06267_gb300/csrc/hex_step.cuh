// Batch-member packs and explicitly rounded arithmetic shared by the step
// kernels of the general-hexahedron path (element stiffness, interface,
// update, layers).  Fields are stored batch-innermost, [node][Bp]; a thread
// moves BB consecutive members of one node as one vector.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace hex {

// BB consecutive batch members of one node, moved as one vector.
template <typename T, int BB>
struct alignas(sizeof(T) * BB) Pack {
  T v[BB];
};

// Explicitly rounded arithmetic: the compiler may not contract or reorder
// these, so a batch member's result is the same for every vector width BB.
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }

// Member-wise operations on a Pack.  FP32 packs of an even width use the
// packed f32x2 instructions (two members per instruction); each lane rounds
// exactly like the scalar form, so results do not depend on the width.
template <typename T, int BB>
constexpr bool packed2() { return std::is_same<T, float>::value && BB % 2 == 0; }

__device__ __forceinline__ float2 sub2_(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// acc += d * x
template <typename T, int BB>
__device__ __forceinline__ void vfma(Pack<T, BB>& acc, T d, const Pack<T, BB>& x) {
  if constexpr (packed2<T, BB>()) {
    const float2 d2 = make_float2(d, d);
#pragma unroll
    for (int b = 0; b < BB; b += 2) {
      float2& a = *reinterpret_cast<float2*>(&acc.v[b]);
      a = __ffma2_rn(d2, *reinterpret_cast<const float2*>(&x.v[b]), a);
    }
  } else {
#pragma unroll
    for (int b = 0; b < BB; ++b) acc.v[b] = fma_(d, x.v[b], acc.v[b]);
  }
}

// d * x
template <typename T, int BB>
__device__ __forceinline__ Pack<T, BB> vmul(T d, const Pack<T, BB>& x) {
  Pack<T, BB> o;
  if constexpr (packed2<T, BB>()) {
    const float2 d2 = make_float2(d, d);
#pragma unroll
    for (int b = 0; b < BB; b += 2)
      *reinterpret_cast<float2*>(&o.v[b]) = __fmul2_rn(d2, *reinterpret_cast<const float2*>(&x.v[b]));
  } else {
#pragma unroll
    for (int b = 0; b < BB; ++b) o.v[b] = mul_(d, x.v[b]);
  }
  return o;
}

// x - y
template <typename T, int BB>
__device__ __forceinline__ Pack<T, BB> vsub(const Pack<T, BB>& x, const Pack<T, BB>& y) {
  Pack<T, BB> o;
  if constexpr (packed2<T, BB>()) {
#pragma unroll
    for (int b = 0; b < BB; b += 2)
      *reinterpret_cast<float2*>(&o.v[b]) =
          sub2_(*reinterpret_cast<const float2*>(&x.v[b]), *reinterpret_cast<const float2*>(&y.v[b]));
  } else {
#pragma unroll
    for (int b = 0; b < BB; ++b) o.v[b] = sub_(x.v[b], y.v[b]);
  }
  return o;
}

// x + y
template <typename T, int BB>
__device__ __forceinline__ Pack<T, BB> vadd(const Pack<T, BB>& x, const Pack<T, BB>& y) {
  Pack<T, BB> o;
  if constexpr (packed2<T, BB>()) {
#pragma unroll
    for (int b = 0; b < BB; b += 2)
      *reinterpret_cast<float2*>(&o.v[b]) =
          __fadd2_rn(*reinterpret_cast<const float2*>(&x.v[b]), *reinterpret_cast<const float2*>(&y.v[b]));
  } else {
#pragma unroll
    for (int b = 0; b < BB; ++b) o.v[b] = add_(x.v[b], y.v[b]);
  }
  return o;
}

template <typename T, int BB>
__device__ __forceinline__ Pack<T, BB> vzero() {
  Pack<T, BB> o;
#pragma unroll
  for (int b = 0; b < BB; ++b) o.v[b] = T(0);
  return o;
}

// vector width: 32 bytes of batch members when the padded batch allows it
template <typename T>
constexpr int vec_width() { return 32 / (int)sizeof(T); }

}  // namespace hex
