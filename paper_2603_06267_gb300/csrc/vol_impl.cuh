// Fused volume step of one box: M^-1 (f - K p) with the sum-factorised GLL
// stiffness of eq. (Wf_2), the PMUT forcing of eq. (f_i) on the z-min plane,
// the SIPG interface residual of the interface element layer, and the
// leapfrog form of the Newmark gamma=1/2, beta=0 corrector/predictor of
// Algorithm 1:  v <- v + dtv * a,  p_out <- p_in + dtp * v.
//
// Layout: one lattice of GLL nodes per box, x fastest, padded row pitch,
// batch members one after another.
//
// Work decomposition: a CTA owns an element-aligned x-y tile of TXE element
// columns x TYE*N rows and marches over a chunk of element layers in z.  A
// thread owns the N nodes of one element along x in one row; PG thread
// groups split the planes of each layer between them (plane c goes to group
// c mod PG), so more warps share one staged tile.  The thread of the last
// element column also owns the box's last x node (a separate, rarely taken
// path).  The N+1 planes of an element layer are staged in shared memory by
// one TMA box load (cp.async.bulk.tensor, zero fill outside the box) with a
// halo of one element on the low x/y side and one node on the high side --
// vertex rows need the neighbouring element, interior rows only their own.
// In FP32 the N planes of v of the layer arrive by a second TMA box into
// the same stage.  Two stages alternate so that the next layer streams in
// while the current one is computed.  The coupling of a vertex plane to the
// layer below is a partial sum carried in registers, so no z halo is loaded.
#pragma once
#include <cstdio>
#include <type_traits>

#include "internal.h"

namespace dgvol {

// ---------------------------------------------------------------------------
// small PTX helpers: mbarrier + TMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `budget` SM clocks (default 2^31, about a
// second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget = 1LL << 31) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}


__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// TMA tensor store shared -> global of a 4-D box (elements outside the
// tensor are not written), and the bulk-group bookkeeping of the issuing thread
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int x, int y, int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of every committed group have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed group has completed (its global writes done)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// vector loads / stores of runs of consecutive elements
// ---------------------------------------------------------------------------
template <typename T, int V> struct Vec;
template <> struct Vec<float, 1> { using t = float; };
template <> struct Vec<float, 2> { using t = float2; };
template <> struct Vec<float, 4> { using t = float4; };
template <> struct Vec<double, 1> { using t = double; };
template <> struct Vec<double, 2> { using t = double2; };

__device__ __forceinline__ void unpack(const float& v, float* o) { o[0] = v; }
__device__ __forceinline__ void unpack(const double& v, double* o) { o[0] = v; }
__device__ __forceinline__ void unpack(const float2& v, float* o) { o[0] = v.x; o[1] = v.y; }
__device__ __forceinline__ void unpack(const float4& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
__device__ __forceinline__ void unpack(const double2& v, double* o) { o[0] = v.x; o[1] = v.y; }

template <typename T, int V>
__device__ __forceinline__ typename Vec<T, V>::t packv(const T* o) {
  typename Vec<T, V>::t v;
  if constexpr (V == 1) v = o[0];
  else if constexpr (V == 2) { v.x = o[0]; v.y = o[1]; }
  else { v.x = o[0]; v.y = o[1]; v.z = o[2]; v.w = o[3]; }
  return v;
}

// load CNT consecutive elements (p aligned to V elements)
template <typename T, int V, int CNT>
__device__ __forceinline__ void vld(const T* __restrict__ p, T* out) {
  static_assert(CNT % V == 0, "run length must be a multiple of the vector width");
  using VT = typename Vec<T, V>::t;
#pragma unroll
  for (int k = 0; k < CNT / V; ++k) unpack(reinterpret_cast<const VT*>(p)[k], out + k * V);
}

template <typename T, int V, int CNT>
__device__ __forceinline__ void vst(T* __restrict__ p, const T* in) {
  static_assert(CNT % V == 0, "run length must be a multiple of the vector width");
  using VT = typename Vec<T, V>::t;
#pragma unroll
  for (int k = 0; k < CNT / V; ++k) reinterpret_cast<VT*>(p)[k] = packv<T, V>(in + k * V);
}

// f(integral_constant<int, I>) for I = B .. E-1, unrolled at compile time
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>());
    static_for<B + 1, E>(f);
  }
}

constexpr int pow2_div(int n) { return (n % 4 == 0) ? 4 : ((n % 2 == 0) ? 2 : 1); }
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr size_t r128(size_t b) { return (b + 127) / 128 * 128; }

// ---------------------------------------------------------------------------
// tile shapes: element columns TXE x element rows TYE per CTA, PG plane
// groups.  Orders 4 and 6 (the workloads' primary and secondary boxes) have
// several shapes the autotuner chooses from; variant 0 is the default.
// ---------------------------------------------------------------------------
// ZR: each thread copies its column of the staged element layer into
// registers once per layer, and the z stencils of its planes and the z carry
// read that copy instead of shared memory (FP32 only); MINB: CTAs per SM;
// RING 3: the p layers in a three-deep ring (v stays two deep), so a p load
// has two layers of work to hide behind; RING 4: the v planes three deep (p
// two), so the v fill of a layer is issued two layers ahead
// TS: the layer's new v and p_next go to shared memory (v in place in its
// stage, p_next into one of two output tiles) and leave by TMA tensor stores,
// one per array and layer, instead of per-thread global stores
template <int A, int B, int C, int Z = 0, int M = 1, int R = 0, int TSV = 0> struct Shape {
  static constexpr int TXE = A, TYE = B, PG = C, MINB = M, RING = R;
  static constexpr bool ZR = Z != 0, TS = TSV != 0;
};
template <typename T, int N, int V> struct TileShape {
  using S = Shape<(N <= 4) ? 32 : 16,
                  (sizeof(T) == 8 && N == 4) ? 2 : ((N <= 2) ? 16 / N : ((N <= 4) ? 4 : (N <= 7 ? 2 : 1))), 1>;
};
template <typename T, int N> struct NumShapes {
  static constexpr int value = (N == 4 || N == 6) ? (sizeof(T) == 4 ? (N == 6 ? 10 : 6) : 4) : 1;
};
// FP32 N=4: 512 / 512 / 512 / 256 threads, register-column 512 / 256 (two CTAs
// per SM); FP64 N=4: 256 / 256 / 128 / 512
template <> struct TileShape<float, 4, 0> { using S = Shape<32, 2, 2>; };
template <> struct TileShape<float, 4, 1> { using S = Shape<32, 4, 1>; };
template <> struct TileShape<float, 4, 2> { using S = Shape<16, 4, 2>; };
template <> struct TileShape<float, 4, 3> { using S = Shape<32, 2, 1>; };
template <> struct TileShape<float, 4, 4> { using S = Shape<32, 4, 1, 1>; };
template <> struct TileShape<float, 4, 5> { using S = Shape<32, 2, 1, 1, 2>; };
template <> struct TileShape<double, 4, 0> { using S = Shape<32, 2, 1>; };
template <> struct TileShape<double, 4, 1> { using S = Shape<16, 4, 1>; };
template <> struct TileShape<double, 4, 2> { using S = Shape<32, 1, 1>; };
template <> struct TileShape<double, 4, 3> { using S = Shape<32, 2, 2>; };
// FP32 N=6: 384 / 576 / 192 / 384 threads, register-column 384 / 192; FP64 N=6:
// 192 / 96 / 192 / 384.  (Two CTAs of half the rows per SM were measured slower
// than one CTA of full rows for both orders.)
template <> struct TileShape<float, 6, 0> { using S = Shape<16, 2, 2>; };
template <> struct TileShape<float, 6, 1> { using S = Shape<16, 2, 3>; };
template <> struct TileShape<float, 6, 2> { using S = Shape<16, 2, 1>; };
template <> struct TileShape<float, 6, 3> { using S = Shape<32, 1, 2>; };
template <> struct TileShape<float, 6, 4> { using S = Shape<16, 2, 2, 1>; };
template <> struct TileShape<float, 6, 5> { using S = Shape<16, 2, 1, 1>; };
template <> struct TileShape<float, 6, 6> { using S = Shape<16, 2, 2, 1, 1, 3>; };
// FP32 N=6 with TMA stores of the outputs: register column, 384 / 576 threads
template <> struct TileShape<float, 6, 7> { using S = Shape<16, 2, 2, 1, 1, 0, 1>; };
template <> struct TileShape<float, 6, 8> { using S = Shape<16, 2, 3, 1, 1, 0, 1>; };
// FP32 N=6, register column, v planes three deep (p two deep): 201 KB
template <> struct TileShape<float, 6, 9> { using S = Shape<16, 2, 2, 1, 1, 4>; };
template <> struct TileShape<double, 6, 0> { using S = Shape<16, 2, 1>; };
template <> struct TileShape<double, 6, 1> { using S = Shape<16, 1, 1>; };
template <> struct TileShape<double, 6, 2> { using S = Shape<8, 4, 1>; };
template <> struct TileShape<double, 6, 3> { using S = Shape<16, 2, 2>; };

template <typename T, int N, int TXE, int TYE, int PG, int RING = 0, bool TS = false>
struct Geo {
  static constexpr int AL = 16 / (int)sizeof(T);                // elements per 16 bytes
  static constexpr int NAL = (N + AL - 1) / AL * AL;            // low x halo rounded up to 16 B
  static constexpr int PAD = NAL - N;
  static constexpr int TYR = TYE * N;                           // owned rows
  static constexpr int BX = (TXE * N + N + 1 + PAD + AL - 1) / AL * AL;   // staged p columns
  static constexpr int BY = TYR + N + 1;                        // staged p rows
  static constexpr int BZ = N + 1;                              // staged p planes (one layer)
  static constexpr int PLANE = BX * BY;
  static constexpr size_t P_BYTES = sizeof(T) * (size_t)BZ * PLANE;
  // v of the owned nodes (+ the box's last x column unless the outputs leave
  // by TMA stores, whose box must hold the owned columns only), N planes,
  // staged in FP32
  static constexpr int BXV = TS ? TXE * N : (TXE * N + 1 + AL - 1) / AL * AL;
  static constexpr int VPLANE = BXV * TYR;
  static constexpr size_t V_BYTES_RAW = sizeof(T) * (size_t)N * VPLANE;
  static constexpr size_t PB = r128(P_BYTES), VBR = r128(V_BYTES_RAW);
  static constexpr int PDEPTH = RING == 3 ? 3 : 2;
  static constexpr int VDEPTH = RING == 4 ? 3 : 2;
  static constexpr bool VTMA = sizeof(T) == 4 && PDEPTH * PB + VDEPTH * VBR + 128 <= 227 * 1024;
  static constexpr size_t V_BYTES = VTMA ? V_BYTES_RAW : 0;
  static constexpr size_t VB = r128(V_BYTES);
  // ring depths: p layers (PST) and v planes (VST, 0 when v is not staged)
  static constexpr int PST = (PDEPTH * PB + (VTMA ? VDEPTH * VB : 0) + 128 <= 227 * 1024) ? PDEPTH : 1;
  static constexpr int VST = VTMA ? VDEPTH : 0;
  static constexpr size_t VBASE = PST * PB;
  // p_next output tiles (two, alternating by layer) of the TMA-store form
  static constexpr size_t OBASE = VBASE + VST * VB;
  static constexpr size_t OB = TS ? VB : 0;
  static constexpr size_t SMEM = PST * PB + VST * VB + 2 * OB + 128;   // + barriers and counters
  static constexpr int NT = TXE * TYR * PG;
  // vector widths: shared-memory runs start at column NAL + tx*N, global runs at ex*N
  static constexpr int VS = cmin(cmin(AL, pow2_div(N)), pow2_div(gcd_c(N, NAL)));
  static constexpr int VG = cmin(AL, pow2_div(N));
  static constexpr int VV = cmin(AL, pow2_div(gcd_c(N, BXV)));   // v runs start at tx*N in a BXV row
  static_assert(NT % 32 == 0 && NT <= 1024, "CTA must be a whole number of warps, at most 1024 threads");
  static_assert(PG >= 1 && PG <= N, "plane groups");
  // TMA: the x coordinates x0 - NAL and x0 (x0 = tile * TXE * N) must be 16-byte aligned
  static_assert((TXE * N * sizeof(T)) % 16 == 0 && (NAL * sizeof(T)) % 16 == 0, "TMA x coordinate misaligned");
  static_assert((BX * sizeof(T)) % 16 == 0 && (BXV * sizeof(T)) % 16 == 0, "TMA box row not a multiple of 16 B");
  static_assert(BX <= 256 && BY <= 256 && BZ <= 256 && BXV <= 256 && TYR <= 256, "TMA box dimension above 256");
  static_assert(SMEM <= 227 * 1024, "tile exceeds shared memory");
  static_assert(!TS || (VTMA && PST == 2 && VST == 2), "TMA stores need the staged v ring");
  static_assert(PST + VST <= 8, "the stage barriers and counters share 128 bytes");
  static_assert(!TS || (TXE * N * sizeof(T)) % 16 == 0, "TMA store box row not a multiple of 16 B");
};

// z stencil of the N owned nodes: sum_q coef[q] * (staged plane q, own column)
template <typename T, int N, int VS, int PLANE>
__device__ __forceinline__ void zsum(const T* __restrict__ S0, int own, const T* coef, T* zs) {
#pragma unroll
  for (int a = 0; a < N; ++a) zs[a] = T(0);
#pragma unroll
  for (int q = 0; q <= N; ++q) {
    T t[N];
    vld<T, VS, N>(S0 + q * PLANE + own, t);
    const T cq = coef[q];
#pragma unroll
    for (int a = 0; a < N; ++a) zs[a] += cq * t[a];
  }
}

// ---------------------------------------------------------------------------
// FP32 stencils.  Every row of the 1D stiffness sums to zero, so
// sum_q c_q p_q = sum_q c_q (p_q - p_ref) for any p_ref.  The FP32 path takes
// p_ref close to the nodes involved (the node itself along y and z, the
// element's first node along x): the summands then have the size of the local
// variation of p rather than of p, and FP32 rounding no longer accumulates
// into a coherent drift over thousands of steps.  The arithmetic is packed
// two lanes wide (f32x2): y and z pair neighbouring owned nodes, x pairs the
// taps of a row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
// a - b, exactly as a subtraction (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// acc[i] += c2 * (t - self) over the owned run (pairs, then a lone last node for odd N)
template <int N, int VS>
__device__ __forceinline__ void run_term(const float* __restrict__ src, float2 c2, const float* self, float2* acc,
                                         float& accT) {
  float t[N];
  vld<float, VS, N>(src, t);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) acc[i] = __ffma2_rn(c2, sub2(f2(t[2 * i], t[2 * i + 1]), f2(self[2 * i], self[2 * i + 1])), acc[i]);
  if constexpr (N % 2 == 1) accT = fmaf(c2.x, t[N - 1] - self[N - 1], accT);
}

// x row: sum_q cq[q] d[q] over q = 0..N with taps in pairs (cq2) and, for even
// N, a lone last tap
template <int N>
__device__ __forceinline__ float row_dot(const float2* cq2, float clast, const float2* d2, float dlast) {
  constexpr int K2 = (N + 1) / 2;
  float2 s = __fmul2_rn(cq2[0], d2[0]);
#pragma unroll
  for (int k = 1; k < K2; ++k) s = __ffma2_rn(cq2[k], d2[k], s);
  float r = s.x + s.y;
  if constexpr (N % 2 == 0) r = fmaf(clast, dlast, r);
  return r;
}

// x part of M^-1 K p of the N owned nodes: xr holds the staged row (left
// element, own element, next vertex); differences to the element's first node
template <int N>
__device__ __forceinline__ void xstencil_f32(const VolArgs<float, N>& A, const float* xr, bool xl, float xiw,
                                             float* acc) {
  constexpr int K2 = (N + 1) / 2;
  const float ref = xr[N];
  const float2 ref2 = f2(ref, ref);
  float2 d2[K2];
#pragma unroll
  for (int k = 0; k < K2; ++k) d2[k] = sub2(f2(xr[N + 2 * k], xr[N + 2 * k + 1]), ref2);
  const float dlast = (N % 2 == 0) ? xr[2 * N] - ref : 0.f;
  float r = row_dot<N>(A.rxq, A.rx[N], d2, dlast);
  if (xl) {
    // for even N the pairs cover q = 0..N-1; the tap q = N is the node itself
    float2 sl = __fmul2_rn(A.lxq[0], sub2(f2(xr[0], xr[1]), ref2));
#pragma unroll
    for (int k = 1; k < K2; ++k) sl = __ffma2_rn(A.lxq[k], sub2(f2(xr[2 * k], xr[2 * k + 1]), ref2), sl);
    r += sl.x + sl.y;
  }
  acc[0] = r * xiw;
#pragma unroll
  for (int a = 1; a < N; ++a) acc[a] = row_dot<N>(A.cxq[a], A.cx[a][N], d2, dlast);
}

// y part: differences to the node itself (self = the owned run of this plane)
template <int N, int VS, int BX>
__device__ __forceinline__ void ystencil_f32(const VolArgs<float, N>& A, const float* __restrict__ P, int own,
                                             const float* self, bool yvert, bool yl, bool yr, float yiw, int yb,
                                             const float2* cyi2, float2* ys, float& ysT) {
  constexpr int NP = N / 2;
  ysT = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) ys[i] = f2(0.f, 0.f);
  if (yvert) {
    if (yl) {
#pragma unroll
      for (int q = 0; q < N; ++q) run_term<N, VS>(P + own + (q - N) * BX, A.ly2[q], self, ys, ysT);
    }
    if (yr) {
#pragma unroll
      for (int q = 1; q <= N; ++q) run_term<N, VS>(P + own + q * BX, A.ry2[q], self, ys, ysT);
    }
    const float2 w2 = f2(yiw, yiw);
#pragma unroll
    for (int i = 0; i < NP; ++i) ys[i] = __fmul2_rn(ys[i], w2);
    ysT *= yiw;
  } else {
#pragma unroll
    for (int q = 0; q <= N; ++q) run_term<N, VS>(P + own + (q - yb) * BX, cyi2[q], self, ys, ysT);
  }
}

// z part from the staged planes (runtime plane c).  ZM: 0 vertex plane
// (carry = lower layer's part), 1 interior plane, 2 top boundary plane.
template <int N, int ZM, int VS, int PLANE>
__device__ __forceinline__ void zstencil_smem_f32(const VolArgs<float, N>& A, const float* __restrict__ S0, int own,
                                                  int c, const float* self, const float* carry, float iw_z,
                                                  float2* zs, float& zsT) {
  constexpr int NP = N / 2;
  zsT = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) zs[i] = f2(0.f, 0.f);
  if constexpr (ZM == 0) {
#pragma unroll
    for (int q = 1; q <= N; ++q) run_term<N, VS>(S0 + q * PLANE + own, A.rz2[q], self, zs, zsT);
  } else if constexpr (ZM == 1) {
#pragma unroll
    for (int q = 0; q <= N; ++q) run_term<N, VS>(S0 + q * PLANE + own, A.cz2[c][q], self, zs, zsT);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) run_term<N, VS>(S0 + q * PLANE + own, A.lz2[q], self, zs, zsT);
  }
  if constexpr (ZM != 1) {
    const float2 w2 = f2(iw_z, iw_z);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const float2 t = (ZM == 0) ? __fadd2_rn(f2(carry[2 * i], carry[2 * i + 1]), zs[i]) : zs[i];
      zs[i] = __fmul2_rn(t, w2);
    }
    if constexpr (N % 2 == 1) zsT = ((ZM == 0 ? carry[N - 1] : 0.f) + zsT) * iw_z;
  }
}

// The register column holds differences to the layer's middle plane R:
// dcol[q] = p_q - p_R of the owned run (dcol[R] = 0, never read).  A full z
// row of the stiffness sums to zero, so sum_q c_q p_q = sum_{q != R} c_q
// dcol[q] exactly; the differences are formed once per layer and shared by
// the thread's planes and the carry, and they have the size of the variation
// of p across one element, as the per-plane differences did.
template <int N> struct ColRef { static constexpr int R = N / 2; };

// the owned run's column differences to plane R, in place
template <int N>
__device__ __forceinline__ void col_to_diff(float (*col)[N]) {
  constexpr int R = ColRef<N>::R;
#pragma unroll
  for (int q = 0; q <= N; ++q) {
    if (q == R) continue;
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 d = sub2(f2(col[q][2 * i], col[q][2 * i + 1]), f2(col[R][2 * i], col[R][2 * i + 1]));
      col[q][2 * i] = d.x;
      col[q][2 * i + 1] = d.y;
    }
    if constexpr (N % 2 == 1) col[q][N - 1] -= col[R][N - 1];
  }
}

// acc += c2 * dcol over the owned run, all in registers
template <int N>
__device__ __forceinline__ void reg_term(const float* dcol, float2 c2, float2* acc, float& accT) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) acc[i] = __ffma2_rn(c2, f2(dcol[2 * i], dcol[2 * i + 1]), acc[i]);
  if constexpr (N % 2 == 1) accT = fmaf(c2.x, dcol[N - 1], accT);
}

// z part from the thread's column differences of the layer, runtime plane c
template <int N, int ZM>
__device__ __forceinline__ void zstencil_col_f32(const VolArgs<float, N>& A, const float (*dcol)[N], int c,
                                                 const float* carry, float iw_z, float2* zs, float& zsT) {
  constexpr int NP = N / 2, R = ColRef<N>::R;
  zsT = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) zs[i] = f2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q <= N; ++q) {
    if (q == R) continue;
    if constexpr (ZM == 0) reg_term<N>(dcol[q], A.rz2[q], zs, zsT);
    else if constexpr (ZM == 1) reg_term<N>(dcol[q], A.cz2[c][q], zs, zsT);
    else reg_term<N>(dcol[q], A.lz2[q], zs, zsT);
  }
  if constexpr (ZM != 1) {
    const float2 w2 = f2(iw_z, iw_z);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const float2 t = (ZM == 0) ? __fadd2_rn(f2(carry[2 * i], carry[2 * i + 1]), zs[i]) : zs[i];
      zs[i] = __fmul2_rn(t, w2);
    }
    if constexpr (N % 2 == 1) zsT = ((ZM == 0 ? carry[N - 1] : 0.f) + zsT) * iw_z;
  }
}

template <int N>
__device__ __forceinline__ void combine_f32(const float* acc, const float2* ys, float ysT, const float2* zs, float zsT,
                                            float* out) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const float2 sm = __fadd2_rn(__fadd2_rn(f2(acc[2 * i], acc[2 * i + 1]), ys[i]), zs[i]);
    out[2 * i] = sm.x;
    out[2 * i + 1] = sm.y;
  }
  if constexpr (N % 2 == 1) out[N - 1] = (acc[N - 1] + ysT) + zsT;
}

// z carry of the next vertex plane (plane N of the layer):
// sum_{q<N} lz[q] (p_q - p_N) of each owned node (FP32 difference form)
template <int N, int VS, int PLANE>
__device__ __forceinline__ void carry_f32(const VolArgs<float, N>& A, const float* __restrict__ S0, int own,
                                          float* carry) {
  constexpr int NP = N / 2;
  float self[N];
  vld<float, VS, N>(S0 + N * PLANE + own, self);
  float2 cs[NP > 0 ? NP : 1];
  float cT = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) cs[i] = f2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < N; ++q) run_term<N, VS>(S0 + q * PLANE + own, A.lz2[q], self, cs, cT);
#pragma unroll
  for (int i = 0; i < NP; ++i) { carry[2 * i] = cs[i].x; carry[2 * i + 1] = cs[i].y; }
  if constexpr (N % 2 == 1) carry[N - 1] = cT;
}

// the same from the column differences in registers
template <int N>
__device__ __forceinline__ void carry_reg_f32(const VolArgs<float, N>& A, const float (*dcol)[N], float* carry) {
  constexpr int NP = N / 2, R = ColRef<N>::R;
  float2 cs[NP > 0 ? NP : 1];
  float cT = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) cs[i] = f2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q <= N; ++q) {
    if (q == R) continue;
    reg_term<N>(dcol[q], A.lz2[q], cs, cT);
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) { carry[2 * i] = cs[i].x; carry[2 * i + 1] = cs[i].y; }
  if constexpr (N % 2 == 1) carry[N - 1] = cT;
}

// Perfectly matched layer.  Does lattice index i (along an axis of ne
// elements) belong to an element of the layer (lo elements at the low side,
// hi at the high side)?
template <int N>
__device__ __forceinline__ bool pml_axis(int i, int ne, int lo, int hi) {
  const int e1 = min(i / N, ne - 1);
  const int e0 = (i % N == 0 && i > 0) ? i / N - 1 : e1;
  return e0 < lo || e1 >= ne - hi;
}

// PML part of the acceleration at node (i, j, k) of batch member b (a node of
// a layer element): beta p + alpha v + gamma psi^{n+1} + M^-1 sum_K (G Phi)_K,
// with psi^{n+1} = psi^{n+1/2} + dt/2 p, and psi^{n+3/2} = psi^{n+1/2} + dt p
// written back.  The initial half step has psi^{1/2} = 0 and Phi^{1/2} = 0:
// only beta p + alpha v.
template <typename T, int N>
__device__ __noinline__ T pml_terms(const VolArgs<T, N>& A, int i, int j, int k, int b, T p, T v, T minv) {
  constexpr int NP = N + 1, NL = NP * NP * NP;
  const T zx = A.zeta[0][i], zy = A.zeta[1][j], zz = A.zeta[2][k];
  T acc = (zx * zy + zy * zz + zz * zx) * p + (zx + zy + zz) * v;
  if (A.pml_init) return acc;
  const long long g = (long long)b * A.bstride + (long long)k * A.pz + (long long)j * A.py + i;
  const T ph = A.psi[g];
  acc += zx * zy * zz * (ph + T(0.5) * A.dtp * p);
  A.psi[g] = ph + A.dtp * p;
  // the node's elements along each axis (two at an element boundary)
  int ex[2], ax[2], ey[2], ay[2], ez[2], az[2];
  auto split = [](int idx, int ne, int* e, int* a) {
    int n = 0;
    if (idx % N == 0) {
      if (idx / N - 1 >= 0) { e[n] = idx / N - 1; a[n] = N; ++n; }
      if (idx / N < ne) { e[n] = idx / N; a[n] = 0; ++n; }
    } else {
      e[n] = idx / N; a[n] = idx % N; ++n;
    }
    return n;
  };
  const int nx = split(i, A.ne0, ex, ax), ny = split(j, A.ne1, ey, ay), nz = split(k, A.ne2, ez, az);
  const T* R = A.rpml + (long long)b * A.rpml_bs;
  T r = T(0);
  for (int c = 0; c < nz; ++c)
    for (int q = 0; q < ny; ++q)
      for (int t = 0; t < nx; ++t) {
        const int slot = A.pml_slot[((long long)ez[c] * A.ne1 + ey[q]) * A.ne0 + ex[t]];
        if (slot >= 0) r += R[(long long)slot * NL + (az[c] * NP + ay[q]) * NP + ax[t]];
      }
  return acc + minv * r;
}

// Row of the tile handled by thread row ty: the TYE vertex rows (element
// boundaries, two-element y stencil) come first so that they fill their own
// warps and the y stencil does not diverge inside a warp.
template <int N, int TYE>
__device__ __forceinline__ int tile_row(int ty) {
  if constexpr (N == 1) {
    return ty;
  } else {
    if (ty < TYE) return ty * N;
    const int i = ty - TYE;
    return (i / (N - 1)) * N + 1 + i % (N - 1);
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <typename T, int N, int TXE, int TYE, int PG, bool ZR, int MINB, bool OPEN, int RING, bool TS>
__global__ void __launch_bounds__(TXE * TYE * N * PG, MINB) vol_kernel(const __grid_constant__ VolArgs<T, N> A) {
  using G = Geo<T, N, TXE, TYE, PG, RING, TS>;
  constexpr bool LATE_CARRY = ZR && MINB == 1;
  static_assert(RING == 0 || G::VTMA, "the three-deep rings are for kernels that stage v");
  static_assert(!ZR || sizeof(T) == 4, "register columns: FP32 only");
  constexpr int BX = G::BX, PLANE = G::PLANE, TYR = G::TYR, NAL = G::NAL, VS = G::VS, VG = G::VG;
  constexpr int BXV = G::BXV, VPLANE = G::VPLANE, VV = G::VV;
  constexpr int PST = G::PST, VST = G::VST;
  constexpr bool VTMA = G::VTMA;
  constexpr bool DIFF = sizeof(T) == 4;    // FP32: difference form, packed arithmetic
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NW = G::NT / 32;
  uint64_t* pbar = reinterpret_cast<uint64_t*>(smem_raw + G::SMEM - 128);   // p stage full
  uint64_t* vbar = pbar + PST;                                                // v stage full
  int* cnt = reinterpret_cast<int*>(pbar + 8);   // warps done with each p stage

  const int tx = threadIdx.x, ty = threadIdx.y, pg = threadIdx.z;
  const int tid = (pg * TYR + ty) * TXE + tx;
  const int ex0 = blockIdx.x * TXE;
  const int x0 = ex0 * N;
  const int y0 = blockIdx.y * TYR;
  const int chunk = blockIdx.z % A.nchunks;
  const int b = blockIdx.z / A.nchunks;
  const int ez0 = chunk * A.layers_per_cta;
  const int ez1 = min(ez0 + A.layers_per_cta, A.ne2);
  const long long boff = (long long)b * A.bstride;
  const T* __restrict__ pin = A.p_in + boff;
  T* __restrict__ pout = A.p_out + boff;
  T* __restrict__ vv = A.v + boff;

  // the last launch of a step advances the run's step counter (read by the
  // PMUT/receiver kernel of the next step, which starts after this one ends)
  if (A.step && tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicAdd(A.step, 1);
  // the TMA destination must be 128-byte aligned
  if (smem_u32(smem_raw) % 128 != 0) {
    if (tid == 0) atomicExch(A.err, 2);
    return;
  }

  const int ex = ex0 + tx;                 // element column
  const int rt = tile_row<N, TYE>(ty);     // row in the tile
  const int j = y0 + rt;                   // lattice row
  const bool active = ex < A.ne0 && j < A.L1;
  const bool xlast = ex == A.ne0 - 1;      // also owns node ne0*N
  const int ey = j / N;
  const int yb = j - ey * N;
  const bool yvert = (yb == 0);
  const bool yl = ey > 0, yr = ey < A.ne1;
  const T yiw = (yl && yr) ? A.iwv : A.iwb;
  T cyi[N + 1];
  float2 cyi2[DIFF ? N + 1 : 1];
#pragma unroll
  for (int q = 0; q <= N; ++q) {
    cyi[q] = yvert ? T(0) : A.cy[yb][q];
    if constexpr (DIFF) cyi2[q] = f2((float)cyi[q], (float)cyi[q]);
  }
  const T iw_y = yvert ? yiw : A.iwa[yb];
  const bool xl = ex > 0;
  const T mscale = T(A.minv_scale);        // 8 / (hx hy hz): M^-1 = mscale / (w_a w_b w_c)
  // absorbing sides: C_ii / M_ii of this row's y sides and of the box's x-min node
  const T abc_y = OPEN ? ((j == 0 ? A.abc[2] : T(0)) + (j == A.L1 - 1 ? A.abc[3] : T(0))) : T(0);
  const T abc_x0 = (OPEN && ex == 0) ? A.abc[0] : T(0);
  const bool pml_y = OPEN && A.has_pml && pml_axis<N>(j, A.ne1, A.pml_lo[1], A.pml_hi[1]);
  auto abc_plane = [&](int k) {   // y and z sides of the nodes of plane k
    return abc_y + (k == 0 ? A.abc[4] : T(0)) + (k == A.L2 - 1 ? A.abc[5] : T(0));
  };
  const T xiw = xl ? A.iwv : A.iwb;        // vertex node ex*N (an element always lies to its right)

  const int r0 = rt + N;                   // staged row of lattice row j
  const int cb = NAL + tx * N;             // staged column of node ex*N
  const int own = r0 * BX + cb;            // staged offset of node ex*N in a p plane
  const int vown = rt * BXV + tx * N;      // staged offset of node ex*N in a v plane
  const long long grow = (long long)j * A.py + (long long)ex * N;   // node ex*N in a plane

  // z carry: sum_q lz[q] p[(ez-1)N + q] of each owned node (plane group 0 owns the vertex planes)
  T carry[N];
  T carryX = T(0);
#pragma unroll
  for (int a = 0; a < N; ++a) carry[a] = T(0);
  if (ez0 > 0 && active && pg == 0) {
    T r[N];
    T rX = T(0);
#pragma unroll
    for (int a = 0; a < N; ++a) r[a] = T(0);
    if constexpr (DIFF) {
      const T* src = pin + (long long)(ez0 * N) * A.pz + grow;     // the vertex plane itself
      vld<T, VG, N>(src, r);
      if (xlast) rX = src[N];
    }
#pragma unroll
    for (int q = 0; q <= N; ++q) {
      T t[N];
      const T* src = pin + (long long)((ez0 - 1) * N + q) * A.pz + grow;
      vld<T, VG, N>(src, t);
#pragma unroll
      for (int a = 0; a < N; ++a) carry[a] += A.lz[q] * (t[a] - r[a]);
      if (xlast) carryX += A.lz[q] * (src[N] - rX);
    }
  }

  // pipeline set-up
  if (tid == 0) {
    for (int s = 0; s < PST; ++s) {
      mbar_init(&pbar[s], 1);
      cnt[s] = 0;
    }
    for (int s = 0; s < VST; ++s) mbar_init(&vbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tmap)) : "memory");
    if constexpr (VTMA) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tmap_v)) : "memory");
  }
  __syncthreads();
  auto issue_p = [&](int ez, int s) {
    mbar_expect_tx(&pbar[s], (uint32_t)G::P_BYTES);
    tma_load_4d(smem_raw + s * G::PB, &A.tmap, &pbar[s], x0 - NAL, y0 - N, ez * N, b);
  };
  auto issue_v = [&](int ez, int s) {
    if constexpr (VTMA) {
      mbar_expect_tx(&vbar[s], (uint32_t)G::V_BYTES);
      tma_load_4d(smem_raw + G::VBASE + s * G::VB, &A.tmap_v, &vbar[s], x0, y0, ez * N, b);
    }
  };
  if (tid == 0) {
    for (int s = 0; s < PST && ez0 + s < ez1; ++s) issue_p(ez0 + s, s);
    for (int s = 0; s < VST && ez0 + s < ez1; ++s) issue_v(ez0 + s, s);
  }

  int it = 0;
  for (int ez = ez0; ez < ez1; ++ez, ++it) {
    const int sp = it % PST, sv = VST ? it % VST : 0;
    const T* S0 = reinterpret_cast<const T*>(smem_raw + sp * G::PB);
    const T* V0 = reinterpret_cast<const T*>(smem_raw + G::VBASE + sv * G::VB);
    // TMA-store form: new v in place in its stage, p_next into this layer's output tile
    T* V0w = reinterpret_cast<T*>(smem_raw + G::VBASE + sv * G::VB);
    T* PO = reinterpret_cast<T*>(smem_raw + G::OBASE + (it & 1) * G::OB);
    const bool last_layer = (ez == A.ne2 - 1);
    const int nplanes = last_layer ? N + 1 : N;
    bool ok = mbar_wait_bounded(&pbar[sp], (uint32_t)((it / PST) & 1));
    if constexpr (VST > 0) ok = ok && mbar_wait_bounded(&vbar[sv], (uint32_t)((it / VST) & 1));
    if (!ok) {
      if (tid == 0) atomicExch(A.err, 1);
      // give the copies in flight a bounded chance to land before leaving
      for (int q = 0; q < PST; ++q) (void)mbar_wait_bounded(&pbar[q], (uint32_t)((it / PST) & 1));
      for (int q = 0; q < VST; ++q) (void)mbar_wait_bounded(&vbar[q], (uint32_t)((it / VST) & 1));
      if constexpr (TS) bulk_wait_all();
      return;
    }
    // ZR: the thread's column of every staged plane of the layer, in registers
    // (the z stencil of all planes and the carry read it); declared outside the
    // active block only where the carry is taken after the stage release
    T colL[LATE_CARRY ? N + 1 : 1][N];
    if (active) {
      T colE[(ZR && !LATE_CARRY) ? N + 1 : 1][N];
      T(*col)[N] = LATE_CARRY ? colL : colE;
      // planes carrying PMUT forcing (z = 0) or interface terms
      auto plane_extras = [&](int k) {
        return (A.has_pmut && k == 0) || (A.iface_k0 >= 0 && k >= A.iface_k0 && k <= A.iface_k0 + N);
      };
      // M^-1 times the extra terms of plane k's owned nodes, from the face arrays
      // assembled for this step: PMUT forcing f (eq. f_i) on z = 0, and
      // -(d_c Rb + [c = top] Ra) of the interface residual on its element layer
      auto plane_extra_vals = [&](int k, T iw_z, T* e) {
        const long long o = (long long)b * A.gbs + (long long)j * A.py + (long long)ex * N;
        T t[N];
#pragma unroll
        for (int a = 0; a < N; ++a) e[a] = T(0);
        if (A.has_pmut && k == 0) {
          vld<T, VG, N>(A.fpm + o, t);
#pragma unroll
          for (int a = 0; a < N; ++a) e[a] += t[a];
        }
        const int idx = k - A.iface_k0;
        if (A.iface_k0 >= 0 && idx >= 0 && idx <= N) {
          vld<T, VG, N>(A.gb + o, t);
          const T d = A.dI[idx];
#pragma unroll
          for (int a = 0; a < N; ++a) e[a] -= d * t[a];
          if (idx == (A.iface_top ? N : 0)) {
            vld<T, VG, N>(A.ga + o, t);
#pragma unroll
            for (int a = 0; a < N; ++a) e[a] -= t[a];
          }
        }
#pragma unroll
        for (int a = 0; a < N; ++a) e[a] *= mscale * ((a == 0) ? xiw : A.iwa[a]) * iw_y * iw_z;
      };
      // the same for the box's last x node (column ex*N + N)
      auto last_extra_val = [&](int k, T iw_z) {
        const long long o = (long long)b * A.gbs + (long long)j * A.py + (long long)ex * N + N;
        T e = T(0);
        if (A.has_pmut && k == 0) e += A.fpm[o];
        const int idx = k - A.iface_k0;
        if (A.iface_k0 >= 0 && idx >= 0 && idx <= N) {
          e -= A.dI[idx] * A.gb[o];
          if (idx == (A.iface_top ? N : 0)) e -= A.ga[o];
        }
        return e * mscale * A.iwb * iw_y * iw_z;
      };
      const bool extras_layer = (A.has_pmut && ez == 0) ||
                                (A.iface_k0 >= 0 && A.iface_k0 <= ez * N + N && A.iface_k0 + N >= ez * N);
      if (extras_layer) {
        // the face rows this thread reads on the layer's planes: start them
        // towards L1 now, so the planes do not wait on DRAM
        const long long o = (long long)b * A.gbs + (long long)j * A.py + (long long)ex * N;
        if (A.has_pmut && ez == 0) { prefetch_l1(A.fpm + o); prefetch_l1(A.fpm + o + N); }
        if (A.iface_k0 >= 0) {
          prefetch_l1(A.gb + o); prefetch_l1(A.gb + o + N);
          prefetch_l1(A.ga + o); prefetch_l1(A.ga + o + N);
        }
      }
      if constexpr (ZR) {
#pragma unroll
        for (int q = 0; q <= N; ++q) vld<T, VS, N>(S0 + q * PLANE + own, col[q]);
        col_to_diff<N>(col);
      }
      // FP32 update of the N owned nodes of plane k from sm = M^-1 K p:
      // a = -sm (+ PMUT / interface terms), v += dtv a, p_out = p + dtp v
      auto commit_f32 = [&](int k, const T* vcur, const T* self, float* sm, T iw_z, T* vn, T* pn) {
        if constexpr (OPEN) {
          // absorbing sides (eq. Wf_4): a -= C/M v with v the predicted velocity v^{n+1/2}
          const T sg = abc_plane(k);
          if (sg != T(0) || abc_x0 != T(0)) {
            sm[0] += (sg + abc_x0) * vcur[0];
#pragma unroll
            for (int a = 1; a < N; ++a) sm[a] += sg * vcur[a];
          }
          if (A.has_pml) {
            const bool yz = pml_y || pml_axis<N>(k, A.ne2, A.pml_lo[2], A.pml_hi[2]);
            for (int a = 0; a < N; ++a) {
              const int i = ex * N + a;
              if (yz || pml_axis<N>(i, A.ne0, A.pml_lo[0], A.pml_hi[0])) {
                const T minv = mscale * ((a == 0) ? xiw : A.iwa[a]) * iw_y * iw_z;
                sm[a] += pml_terms<T, N>(A, i, j, k, b, self[a], vcur[a], minv);
              }
            }
          }
        }
        if (extras_layer && plane_extras(k)) {
          T e[N];
          plane_extra_vals(k, iw_z, e);
#pragma unroll
          for (int a = 0; a < N; ++a) sm[a] -= e[a];
        }
        const float2 ndtv = f2(-A.dtv, -A.dtv), dtp = f2(A.dtp, A.dtp);
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
          const float2 v2 = __ffma2_rn(ndtv, f2(sm[2 * i], sm[2 * i + 1]), f2(vcur[2 * i], vcur[2 * i + 1]));
          const float2 p2 = __ffma2_rn(dtp, v2, f2(self[2 * i], self[2 * i + 1]));
          vn[2 * i] = v2.x; vn[2 * i + 1] = v2.y;
          pn[2 * i] = p2.x; pn[2 * i + 1] = p2.y;
        }
        if constexpr (N % 2 == 1) {
          vn[N - 1] = vcur[N - 1] - A.dtv * sm[N - 1];
          pn[N - 1] = self[N - 1] + A.dtp * vn[N - 1];
        }
      };
      // one plane of the layer for the N owned nodes; ZM selects the z rows:
      // 0 vertex plane (carried lower part + own layer), 1 interior plane c,
      // 2 top boundary plane of the box
      auto plane = [&](auto zm, int c) {
        constexpr int ZM = decltype(zm)::value;
        const T* P = S0 + c * PLANE;
        const int k = ez * N + c;
        T vcur[N];
        if constexpr (VTMA && ZM != 2) {
          vld<T, VV, N>(V0 + c * VPLANE + vown, vcur);
        } else {
          vld<T, VG, N>(vv + (long long)k * A.pz + grow, vcur);
        }
        // staged row of lattice row j: columns cb-N .. cb+N-1
        T xr[2 * N + 1];
        vld<T, VS, N>(P + own - N, xr);
        vld<T, VS, N>(P + own, xr + N);
        xr[2 * N] = P[own + N];
        T vn[N], pn[N];
        T iw_z;
        if constexpr (ZM == 0) iw_z = (ez > 0) ? A.iwv : A.iwb;
        else if constexpr (ZM == 1) iw_z = A.iwa[c];
        else iw_z = A.iwb;
        if constexpr (DIFF) {
          float acc[N], sm[N];
          float2 ys[N / 2 > 0 ? N / 2 : 1], zs[N / 2 > 0 ? N / 2 : 1];
          float ysT, zsT;
          xstencil_f32<N>(A, xr, xl, xiw, acc);
          ystencil_f32<N, VS, BX>(A, P, own, xr + N, yvert, yl, yr, yiw, yb, cyi2, ys, ysT);
          if constexpr (ZR) zstencil_col_f32<N, ZM>(A, col, c, carry, iw_z, zs, zsT);
          else zstencil_smem_f32<N, ZM, VS, PLANE>(A, S0, own, c, xr + N, carry, iw_z, zs, zsT);
          combine_f32<N>(acc, ys, ysT, zs, zsT, sm);
          commit_f32(k, vcur, xr + N, sm, iw_z, vn, pn);
        } else {
          T acc[N];
          // x stencil
          {
            T l = T(0), r = T(0);
            if (xl) {
#pragma unroll
              for (int q = 0; q <= N; ++q) l += A.lx[q] * xr[q];
            }
#pragma unroll
            for (int q = 0; q <= N; ++q) r += A.rx[q] * xr[N + q];
            acc[0] = (l + r) * xiw;
          }
#pragma unroll
          for (int a = 1; a < N; ++a) {
            T s2 = T(0);
#pragma unroll
            for (int q = 0; q <= N; ++q) s2 += A.cx[a][q] * xr[N + q];
            acc[a] = s2;
          }
          // y stencil
          if (yvert) {
            T ylv[N], yrv[N];
#pragma unroll
            for (int a = 0; a < N; ++a) { ylv[a] = T(0); yrv[a] = T(0); }
            if (yl) {
#pragma unroll
              for (int q = 0; q <= N; ++q) {
                T t[N];
                vld<T, VS, N>(P + own + (q - N) * BX, t);
#pragma unroll
                for (int a = 0; a < N; ++a) ylv[a] += A.ly[q] * t[a];
              }
            }
            if (yr) {
#pragma unroll
              for (int q = 0; q <= N; ++q) {
                T t[N];
                vld<T, VS, N>(P + own + q * BX, t);
#pragma unroll
                for (int a = 0; a < N; ++a) yrv[a] += A.ry[q] * t[a];
              }
            }
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a] += (ylv[a] + yrv[a]) * yiw;
          } else {
#pragma unroll
            for (int q = 0; q <= N; ++q) {
              T t[N];
              vld<T, VS, N>(P + own + (q - yb) * BX, t);
#pragma unroll
              for (int a = 0; a < N; ++a) acc[a] += cyi[q] * t[a];
            }
          }
          // z stencil: own column over the staged planes of the layer
          T zs[N];
          if constexpr (ZM == 0) {
            zsum<T, N, VS, PLANE>(S0, own, A.rz, zs);
#pragma unroll
            for (int a = 0; a < N; ++a) zs[a] = (carry[a] + zs[a]) * iw_z;
          } else if constexpr (ZM == 1) {
            zsum<T, N, VS, PLANE>(S0, own, A.cz[c], zs);
          } else {
            zsum<T, N, VS, PLANE>(S0, own, A.lz, zs);
#pragma unroll
            for (int a = 0; a < N; ++a) zs[a] *= iw_z;
          }
          // update: a = -(M^-1 K p) - C/M v (+ extras), v += dtv a, p_out = p + dtp v
          const T sg = OPEN ? abc_plane(k) : T(0);
          T ext[N];
#pragma unroll
          for (int a = 0; a < N; ++a) ext[a] = T(0);
          if (extras_layer && plane_extras(k)) plane_extra_vals(k, iw_z, ext);
#pragma unroll
          for (int a = 0; a < N; ++a) {
            T accum = -(acc[a] + zs[a]);
            if constexpr (OPEN) {
              accum -= (sg + (a == 0 ? abc_x0 : T(0))) * vcur[a];
              if (A.has_pml && (pml_y || pml_axis<N>(k, A.ne2, A.pml_lo[2], A.pml_hi[2]) ||
                                pml_axis<N>(ex * N + a, A.ne0, A.pml_lo[0], A.pml_hi[0]))) {
                const T minv = mscale * ((a == 0) ? xiw : A.iwa[a]) * iw_y * iw_z;
                accum -= pml_terms<T, N>(A, ex * N + a, j, k, b, xr[N + a], vcur[a], minv);
              }
            }
            accum += ext[a];
            vn[a] = vcur[a] + A.dtv * accum;
            pn[a] = xr[N + a] + A.dtp * vn[a];
          }
        }
        if constexpr (TS && ZM != 2) {
          vst<T, VV, N>(V0w + c * VPLANE + vown, vn);
          vst<T, VV, N>(PO + c * VPLANE + vown, pn);
        } else {
          vst<T, VG, N>(vv + (long long)k * A.pz + grow, vn);
          vst<T, VG, N>(pout + (long long)k * A.pz + grow, pn);
        }
      };
      // the box's last x node (column cb+N), owned by the last element column
      auto plane_last_x = [&](int c) {
        const T* P = S0 + c * PLANE;
        const int k = ez * N + c;
        const int col = own + N;
        const T self = DIFF ? P[col] : T(0);
        T x = T(0);
#pragma unroll
        for (int q = 0; q <= N; ++q) x += A.lx[q] * (P[own + q] - self);
        x *= A.iwb;
        T y;
        if (yvert) {
          T l = T(0), r = T(0);
          if (yl) {
#pragma unroll
            for (int q = 0; q <= N; ++q) l += A.ly[q] * (P[col + (q - N) * BX] - self);
          }
          if (yr) {
#pragma unroll
            for (int q = 0; q <= N; ++q) r += A.ry[q] * (P[col + q * BX] - self);
          }
          y = (l + r) * yiw;
        } else {
          y = T(0);
#pragma unroll
          for (int q = 0; q <= N; ++q) y += cyi[q] * (P[col + (q - yb) * BX] - self);
        }
        T z = T(0), iw_z;
        if (c == 0) {
#pragma unroll
          for (int q = 0; q <= N; ++q) z += A.rz[q] * (S0[q * PLANE + col] - self);
          iw_z = (ez > 0) ? A.iwv : A.iwb;
          z = (carryX + z) * iw_z;
        } else if (c < N) {
#pragma unroll
          for (int q = 0; q <= N; ++q) z += A.cz[c][q] * (S0[q * PLANE + col] - self);
          iw_z = A.iwa[c];
        } else {
#pragma unroll
          for (int q = 0; q <= N; ++q) z += A.lz[q] * (S0[q * PLANE + col] - self);
          iw_z = A.iwb;
          z *= iw_z;
        }
        T accum = -(x + y + z);
        if (extras_layer && plane_extras(k)) accum += last_extra_val(k, iw_z);
        T* vp = vv + (long long)k * A.pz + grow + N;
        // TMA-store form: the column lies in the tile's store box only when the
        // tile is ragged (an inactive column follows); otherwise it is the box's
        // right neighbour and goes to global memory directly
        const bool in_box = TS && c < N && tx < TXE - 1;
        T vo;
        if constexpr (VTMA) vo = (c < N && (!TS || tx < TXE - 1)) ? V0[c * VPLANE + vown + N] : *vp;
        else vo = *vp;
        if constexpr (OPEN) {
          accum -= (abc_plane(k) + A.abc[1]) * vo;
          if (A.has_pml) accum -= pml_terms<T, N>(A, ex * N + N, j, k, b, P[col], vo, mscale * A.iwb * iw_y * iw_z);
        }
        const T vn = vo + A.dtv * accum;
        if (in_box) {
          V0w[c * VPLANE + vown + N] = vn;
          PO[c * VPLANE + vown + N] = P[col] + A.dtp * vn;
        } else {
          *vp = vn;
          pout[(long long)k * A.pz + grow + N] = P[col] + A.dtp * vn;
        }
      };
      if constexpr (ZR && N <= 4) {
        // register-column kernels of order <= 4: every plane index is a
        // compile-time constant, so its z coefficients and offsets are immediate
        // operands (order 4: 2.85 against 3.03 ms per config-4 launch; at order
        // 6 the seven plane copies double the code to 83 KB and the kernel runs
        // a third slower, so it keeps the runtime plane loop)
        static_for<0, N + 1>([&](auto cc) {
          constexpr int C = decltype(cc)::value;
          if (C % PG == pg && C < nplanes) {
            plane(std::integral_constant<int, C == 0 ? 0 : (C < N ? 1 : 2)>(), C);
            if (xlast) plane_last_x(C);
          }
        });
      } else {
        for (int c = pg; c < nplanes; c += PG) {
          if (c == 0) plane(std::integral_constant<int, 0>(), 0);
          else if (c < N) plane(std::integral_constant<int, 1>(), c);
          else plane(std::integral_constant<int, 2>(), N);
          if (xlast) plane_last_x(c);
        }
      }
      // carry for the vertex plane (ez+1)*N (register-column kernels of one
      // CTA per SM: after the stage is released, below, since it reads
      // registers only -- the stage's last reader releases it sooner; measured
      // 0.4 % faster for order 6, 3.5 % slower for the two-CTA order-4 tile)
      if (pg == 0) {
        if constexpr (ZR && !LATE_CARRY) carry_reg_f32<N>(A, col, carry);
        if constexpr (!ZR) {
          if constexpr (DIFF) carry_f32<N, VS, PLANE>(A, S0, own, carry);
          else zsum<T, N, VS, PLANE>(S0, own, A.lz, carry);
        }
        if (xlast) {
          const T self = DIFF ? S0[N * PLANE + own + N] : T(0);
          carryX = T(0);
#pragma unroll
          for (int q = 0; q <= N; ++q) carryX += A.lz[q] * (S0[q * PLANE + own + N] - self);
        }
      }
    }
    // release the layer's stages: the last warp to finish reading them issues their next
    // load, so warps with more work in this layer (vertex rows, the z carry)
    // hold up the others only when the ring runs dry
    // TMA-store form: the outputs this thread wrote to shared memory become
    // visible to the async proxy before the counter hands them to the store
    if constexpr (TS) fence_proxy_async_smem();
    __syncwarp();
    if ((tid & 31) == 0) {
      __threadfence_block();
      if (atomicAdd(&cnt[sp], 1) == NW - 1) {
        cnt[sp] = 0;
        __threadfence_block();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if constexpr (TS) {
          // the layer's planes ez*N .. ez*N+N-1 of v (in place in its stage) and
          // p_next; the stage is refilled only once the stores have read it
          tma_store_4d(&A.tmap_v, V0w, x0, y0, ez * N, b);
          tma_store_4d(&A.tmap_pst, PO, x0, y0, ez * N, b);
          bulk_commit();
          bulk_wait_read_all();
        }
        if (ez + PST < ez1) issue_p(ez + PST, sp);
        if (ez + VST < ez1) issue_v(ez + VST, sv);
      }
    }
    if constexpr (LATE_CARRY) {
      if (active && pg == 0) carry_reg_f32<N>(A, colL, carry);
    }
  }
  // stores issued by this thread have completed before the CTA leaves
  if constexpr (TS) bulk_wait_all();
}

template <typename T, int N>
VolArgs<T, N> make_args(const VolSpec& s) {
  VolArgs<T, N> a;
  a.tmap = *s.tmap;
  if (s.tmap_v) a.tmap_v = *s.tmap_v;
  if (s.tmap_pst) a.tmap_pst = *s.tmap_pst;
  a.err = s.err;
  a.step = s.step;
  a.p_in = static_cast<const T*>(s.p_in);
  a.p_out = static_cast<T*>(s.p_out);
  a.v = static_cast<T*>(s.v);
  a.bstride = s.bstride;
  a.L0 = s.L[0]; a.L1 = s.L[1]; a.L2 = s.L[2];
  a.ne0 = s.ne[0]; a.ne1 = s.ne[1]; a.ne2 = s.ne[2];
  a.py = s.py; a.pz = s.pz;
  a.dtv = T(s.dtv); a.dtp = T(s.dtp);
  for (int p = 0; p <= N; ++p) {
    for (int q = 0; q <= N; ++q) {
      a.cx[p][q] = T(s.c[0][p][q]);
      a.cy[p][q] = T(s.c[1][p][q]);
      a.cz[p][q] = T(s.c[2][p][q]);
    }
    a.lx[p] = T(s.l[0][p]); a.rx[p] = T(s.r[0][p]);
    a.ly[p] = T(s.l[1][p]); a.ry[p] = T(s.r[1][p]);
    a.lz[p] = T(s.l[2][p]); a.rz[p] = T(s.r[2][p]);
    a.iwa[p] = T(s.iwa[p]);
    a.dI[p] = T(s.dI[p]);
  }
  for (int p = 0; p <= N; ++p) {
    for (int k = 0; k < (N + 1) / 2; ++k) {
      // taps past q = N (odd N) do not occur: the pairs end at q = N
      a.cxq[p][k] = make_float2((float)s.c[0][p][2 * k], (float)s.c[0][p][2 * k + 1]);
    }
    for (int q = 0; q <= N; ++q) a.cz2[p][q] = make_float2((float)s.c[2][p][q], (float)s.c[2][p][q]);
    a.ly2[p] = make_float2((float)s.l[1][p], (float)s.l[1][p]);
    a.ry2[p] = make_float2((float)s.r[1][p], (float)s.r[1][p]);
    a.lz2[p] = make_float2((float)s.l[2][p], (float)s.l[2][p]);
    a.rz2[p] = make_float2((float)s.r[2][p], (float)s.r[2][p]);
  }
  for (int k = 0; k < (N + 1) / 2; ++k) {
    a.lxq[k] = make_float2((float)s.l[0][2 * k], (float)s.l[0][2 * k + 1]);
    a.rxq[k] = make_float2((float)s.r[0][2 * k], (float)s.r[0][2 * k + 1]);
  }
  for (int q = 0; q < 6; ++q) a.abc[q] = T(s.abc[q]);
  a.has_abc = s.has_abc;
  a.has_pml = s.has_pml;
  a.pml_init = s.pml_init;
  for (int d = 0; d < 3; ++d) {
    a.zeta[d] = static_cast<const T*>(s.zeta[d]);
    a.pml_lo[d] = s.pml_lo[d];
    a.pml_hi[d] = s.pml_hi[d];
  }
  a.psi = static_cast<T*>(s.psi);
  a.rpml = static_cast<const T*>(s.rpml);
  a.pml_slot = s.pml_slot;
  a.rpml_bs = s.rpml_bs;
  a.iwv = T(s.iwv); a.iwb = T(s.iwb);
  a.minv_scale = s.minv_scale;
  a.has_pmut = s.has_pmut;
  a.fpm = static_cast<const T*>(s.fpm);
  a.iface_k0 = s.iface_k0; a.iface_top = s.iface_top;
  a.ga = static_cast<const T*>(s.ga); a.gb = static_cast<const T*>(s.gb);
  a.gbs = s.gbs;
  return a;
}

template <typename T, int N, int V, bool OPEN>
cudaError_t launch_v(const VolSpec& s, int batch, cudaStream_t st) {
  using SH = typename TileShape<T, N, V>::S;
  constexpr int TXE = SH::TXE, TYE = SH::TYE, PG = SH::PG;
  using G = Geo<T, N, TXE, TYE, PG, SH::RING, SH::TS>;
  if (!s.tmap || !s.err) return cudaErrorInvalidValue;
  if (G::VTMA && !s.tmap_v) return cudaErrorInvalidValue;
  if (SH::TS && !s.tmap_pst) return cudaErrorInvalidValue;
  VolArgs<T, N> a = make_args<T, N>(s);
  int layers = s.layers_per_cta;
  const int gx = (s.ne[0] + TXE - 1) / TXE;
  const int gy = (s.L[1] + G::TYR - 1) / G::TYR;
  if (layers <= 0) {
    // enough CTAs to fill every SM a few times over
    const long long cols = (long long)gx * gy * batch;
    layers = s.ne[2];
    while (layers > 1 && cols * ((s.ne[2] + layers - 1) / layers) < 4 * 152) layers = (layers + 1) / 2;
  }
  a.layers_per_cta = layers;
  a.nchunks = (s.ne[2] + layers - 1) / layers;
  auto kern = vol_kernel<T, N, TXE, TYE, PG, SH::ZR, SH::MINB, OPEN, SH::RING, SH::TS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(gx, gy, a.nchunks * batch);
  dim3 block(TXE, G::TYR, PG);
  if (s.shape_out) {
    const int sh[8] = {(int)grid.x, (int)grid.y, (int)grid.z, (int)block.x, (int)block.y, (int)block.z, layers, a.nchunks};
    for (int i = 0; i < 8; ++i) s.shape_out[i] = sh[i];
  }
  kern<<<grid, block, G::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, bool OPEN>
cudaError_t launch_n(const VolSpec& s, int batch, cudaStream_t st) {
  if constexpr (NumShapes<T, N>::value > 1) {
    switch (s.tile) {
      case 0: return launch_v<T, N, 0, OPEN>(s, batch, st);
      case 1: return launch_v<T, N, 1, OPEN>(s, batch, st);
      case 2: return launch_v<T, N, 2, OPEN>(s, batch, st);
      case 3: return launch_v<T, N, 3, OPEN>(s, batch, st);
      case 4: if constexpr (NumShapes<T, N>::value > 4) return launch_v<T, N, 4, OPEN>(s, batch, st); break;
      case 5: if constexpr (NumShapes<T, N>::value > 5) return launch_v<T, N, 5, OPEN>(s, batch, st); break;
      case 6: if constexpr (NumShapes<T, N>::value > 6) return launch_v<T, N, 6, OPEN>(s, batch, st); break;
      case 7: if constexpr (NumShapes<T, N>::value > 7) return launch_v<T, N, 7, OPEN>(s, batch, st); break;
      case 8: if constexpr (NumShapes<T, N>::value > 8) return launch_v<T, N, 8, OPEN>(s, batch, st); break;
      case 9: if constexpr (NumShapes<T, N>::value > 9) return launch_v<T, N, 9, OPEN>(s, batch, st); break;
      default: break;
    }
    return cudaErrorInvalidValue;
  } else {
    if (s.tile != 0) return cudaErrorInvalidValue;
    return launch_v<T, N, 0, OPEN>(s, batch, st);
  }
}

template <typename T, int N, int V>
void box_v(unsigned box[3], unsigned vbox[3]) {
  using SH = typename TileShape<T, N, V>::S;
  using G = Geo<T, N, SH::TXE, SH::TYE, SH::PG, SH::RING, SH::TS>;
  box[0] = G::BX;
  box[1] = G::BY;
  box[2] = G::BZ;
  vbox[0] = G::VTMA ? G::BXV : 0;
  vbox[1] = G::VTMA ? G::TYR : 0;
  vbox[2] = G::VTMA ? N : 0;
}

template <typename T, int N>
int box_n(int tile, unsigned box[3], unsigned vbox[3]) {
  box[0] = box[1] = box[2] = 0;
  vbox[0] = vbox[1] = vbox[2] = 0;
  if (tile < 0 || tile >= NumShapes<T, N>::value) return 0;
  if constexpr (NumShapes<T, N>::value > 1) {
    switch (tile) {
      case 0: box_v<T, N, 0>(box, vbox); break;
      case 1: box_v<T, N, 1>(box, vbox); break;
      case 2: box_v<T, N, 2>(box, vbox); break;
      case 3: box_v<T, N, 3>(box, vbox); break;
      case 4: if constexpr (NumShapes<T, N>::value > 4) box_v<T, N, 4>(box, vbox); break;
      case 5: if constexpr (NumShapes<T, N>::value > 5) box_v<T, N, 5>(box, vbox); break;
      case 6: if constexpr (NumShapes<T, N>::value > 6) box_v<T, N, 6>(box, vbox); break;
      case 7: if constexpr (NumShapes<T, N>::value > 7) box_v<T, N, 7>(box, vbox); break;
      case 8: if constexpr (NumShapes<T, N>::value > 8) box_v<T, N, 8>(box, vbox); break;
      default: if constexpr (NumShapes<T, N>::value > 9) box_v<T, N, 9>(box, vbox); break;
    }
  } else {
    box_v<T, N, 0>(box, vbox);
  }
  return NumShapes<T, N>::value;
}

// Host entry points of one precision (instantiated in vol_f32.cu / vol_f64.cu)
template <typename T>
int tma_box(int N, int tile, unsigned box[3], unsigned vbox[3]) {
  switch (N) {
    case 1: return box_n<T, 1>(tile, box, vbox);
    case 2: return box_n<T, 2>(tile, box, vbox);
    case 3: return box_n<T, 3>(tile, box, vbox);
    case 4: return box_n<T, 4>(tile, box, vbox);
    case 5: return box_n<T, 5>(tile, box, vbox);
    case 6: return box_n<T, 6>(tile, box, vbox);
    case 7: return box_n<T, 7>(tile, box, vbox);
    case 8: return box_n<T, 8>(tile, box, vbox);
    default: box[0] = box[1] = box[2] = 0; vbox[0] = vbox[1] = vbox[2] = 0; return 0;
  }
}

}  // namespace dgvol

template <typename T, bool OPEN>
cudaError_t launch_vol_flag(const VolSpec& s, int batch, cudaStream_t st) {
  using namespace dgvol;
  switch (s.N) {
    case 1: return launch_n<T, 1, OPEN>(s, batch, st);
    case 2: return launch_n<T, 2, OPEN>(s, batch, st);
    case 3: return launch_n<T, 3, OPEN>(s, batch, st);
    case 4: return launch_n<T, 4, OPEN>(s, batch, st);
    case 5: return launch_n<T, 5, OPEN>(s, batch, st);
    case 6: return launch_n<T, 6, OPEN>(s, batch, st);
    case 7: return launch_n<T, 7, OPEN>(s, batch, st);
    case 8: return launch_n<T, 8, OPEN>(s, batch, st);
    default: return cudaErrorInvalidValue;
  }
}
