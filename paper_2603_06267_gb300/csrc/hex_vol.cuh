// Element stiffness of the general-hexahedron step, eq. (Wf_2): the kernel
// template and its launch variants.  Instantiated per precision in
// hex_vol_f32.cu and hex_vol_f64.cu.
#pragma once

#include <cuda_runtime.h>

#include "hex_geom.h"
#include "hex_step.cuh"

namespace {

// cp.async (sm_80+): asynchronous global -> shared copies, completed by
// commit/wait groups; they keep no registers busy while in flight.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// copy of `bytes` (4, 8, 16 or 32; both addresses aligned to it)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  if constexpr (BYTES == 32) {
    cp_async16(smem, gmem);
    cp_async16(static_cast<char*>(smem) + 16, static_cast<const char*>(gmem) + 16);
  } else if constexpr (BYTES == 16) {
    cp_async16(smem, gmem);
  } else if constexpr (BYTES == 8) {
    cp_async8(smem, gmem);
  } else {
    static_assert(BYTES == 4, "cp.async size");
    cp_async4(smem, gmem);
  }
}

}  // namespace

namespace hex {

// Element stiffness of eq. (Wf_2), sum-factorised along element lines.
// A CTA takes E elements and BB batch members at a time; each element has
// n^2 threads, and thread q of an element owns the x-line (b, c), the y-line
// (a, c) and the z-line (a, b) with (., .) = (q mod n, q div n):
//   A: x- and y-lines: grad^_x u, grad^_y u of their line in difference form
//      sum_m D_am (u_m - u_0) with the line's first node as reference (exact
//      for constants in any precision; rounding scales with the variation
//      along the line, not with u) -> smem
//   B: z-line: grad^_z u in registers, then F = G grad^ u at its nodes with
//      the geometric factors G; F_x, F_y -> smem, F_z kept for D
//   C: x-lines: D^T F_x -> R_x; y-lines: D^T F_y -> R_y
//   D: z-line: r = R_x + R_y + D^T F_z -> the element's residual slots.
// Every line contraction uses the even-odd split of D (eo_line); its
// coefficients are indexed by compile-time indices only (uniform across the
// warp), and the per-member arithmetic is the same for every BB.
//
// Launch variants (flags FL) trade registers and shared memory for resident
// CTAs; all of them do the same arithmetic in the same order, so their
// results agree bit for bit:
//   VOL_LEAN  F_z goes to the z-line's own entries of the u buffer instead
//             of registers, R_x replaces F_x in place
//   VOL_GSM   geometric factors staged in shared memory once per CTA
//             (otherwise read through the read-only cache at each chunk)
//   VOL_DB    two u buffers: the next chunk's gather is in flight while the
//             current one is computed
enum : int { VOL_LEAN = 1, VOL_GSM = 2, VOL_DB = 4 };

template <int N, int E_>
struct VolTeam {
  static constexpr int n = N + 1, nl = n * n * n, line = n * n;
  static constexpr int E = E_;                                     // elements per CTA
  static constexpr int threads = (E * line + 31) / 32 * 32;
};

// E0: as many elements as fill 128 threads
template <int N>
constexpr int vol_e0() {
  constexpr int line = (N + 1) * (N + 1);
  return line >= 128 ? 1 : 128 / line;
}

// E1: the element count (at most 256 threads) that leaves the smallest share
// of idle lanes in the last warp; E0 when it is as good
template <int N>
constexpr int vol_e1() {
  constexpr int line = (N + 1) * (N + 1);
  int best = vol_e0<N>();
  for (int e = 1; e * line <= 256; ++e) {
    const long long te = (e * line + 31) / 32 * 32, tb = (best * line + 31) / 32 * 32;
    if ((te - e * line) * tb < (tb - best * line) * te) best = e;
  }
  return best;
}

template <typename T, int BB, int N, int E, int FL>
constexpr size_t vol_geo_off() {
  constexpr size_t planes = (FL & VOL_DB) ? 4 : 3;
  return (planes * sizeof(T) * BB * (size_t)VolTeam<N, E>::nl * E + 15) / 16 * 16;
}

// shared memory: u buffer(s) (the current one then holds F_z or R_x), the
// x/y gradients (then F_x, F_y, R_x/R_y), and the CTA's geometric factors
template <typename T, int BB, int N, int E, int FL>
constexpr size_t vol_smem() {
  return vol_geo_off<T, BB, N, E, FL>() +
         ((FL & VOL_GSM) ? sizeof(T) * 6 * (size_t)((VolTeam<N, E>::nl + 3) / 4 * 4) * E : 0);
}

// resident CTAs per SM the lean variants ask the register allocator for: as
// many as the shared memory allows (228 KB per SM, 1 KB reserved per CTA),
// capped so that a thread keeps at least 80 registers; the other variants
// leave the allocator free
template <typename T, int BB, int N, int E, int FL>
constexpr int vol_min_blocks() {
  if (!(FL & VOL_LEAN)) return 1;
  constexpr long long by_smem = 233472LL / ((long long)vol_smem<T, BB, N, E, FL>() + 1024);
  constexpr long long by_regs = 65536LL / (80LL * VolTeam<N, E>::threads);
  constexpr long long b = by_smem < by_regs ? by_smem : by_regs;
  return b < 1 ? 1 : (int)b;
}

// A shared array of packs stored as planes of 16-byte entries (members
// [0, H), [H, 2H), ...): a warp's 16-byte accesses to consecutive entries are
// then contiguous and free of bank conflicts.
template <typename T, int BB>
struct SPlanes {
  static constexpr int H = (int)(sizeof(T) * BB > 16 ? 16 / sizeof(T) : BB);   // members per entry
  static constexpr int NPL = BB / H;                                           // planes
  using P = Pack<T, BB>;
  using Half = Pack<T, H>;
  T* base;
  int count;
  __device__ __forceinline__ T* ptr(int pl, int k) const { return base + ((long long)pl * count + k) * H; }
  __device__ __forceinline__ P ld(int k) const {
    P o;
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) *reinterpret_cast<Half*>(&o.v[pl * H]) = *reinterpret_cast<const Half*>(ptr(pl, k));
    return o;
  }
  __device__ __forceinline__ void st(int k, const P& x) const {
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) *reinterpret_cast<Half*>(ptr(pl, k)) = *reinterpret_cast<const Half*>(&x.v[pl * H]);
  }
};

// One line contraction out_a = sum_m C_am l_m with C = D (TR false: the
// reference gradient, in difference form: l_m - l_0 replaces l_m) or C = D^T
// (TR true), by its even-odd split.  Both matrices are centro-antisymmetric
// on GLL nodes (C_{n-1-a, n-1-m} = -C_am), so with h = n / 2,
// s_m = l_m + l_{n-1-m} and d_m = l_m - l_{n-1-m} (m < h):
//   P_a = sum_{m<h} ea_am d_m,  Q_a = sum_{m<h} eb_am s_m (+ eb_ah l_h, odd n)
//   out_a = P_a + Q_a,  out_{n-1-a} = P_a - Q_a  (a < h)
//   out_h = sum_{m<h} em_m d_m  (odd n; C_hh = 0)
// with ea = (C_am - C_{a,n-1-m}) / 2, eb = (C_am + C_{a,n-1-m}) / 2,
// eb_ah = C_ah, em_m = C_hm: about 3/4 of the direct n^2 multiply-adds.  In
// the difference form l_0 = 0, so s_0 = l_{n-1}, d_0 = -l_{n-1}.  Outputs go
// to emit(a, value) as they are formed (a compile-time index once unrolled).
template <typename T, int BB, int n, bool TR, class F>
__device__ __forceinline__ void eo_line(const HexVolArgs<T>& A, Pack<T, BB> (&l)[n], F&& emit) {
  using P = Pack<T, BB>;
  constexpr int h = n / 2, t = TR ? 1 : 0, m0 = TR ? 0 : 1;
  if constexpr (!TR) {
#pragma unroll
    for (int m = n - 1; m > 0; --m) l[m] = vsub(l[m], l[0]);
  }
  P s[h], d[h];
#pragma unroll
  for (int m = m0; m < h; ++m) {
    s[m] = vadd(l[m], l[n - 1 - m]);
    d[m] = vsub(l[m], l[n - 1 - m]);
  }
#pragma unroll
  for (int a = 0; a < h; ++a) {
    P p, q;
    if constexpr (TR) {
      p = vmul(T(A.ea[t][a][0]), d[0]);
      q = vmul(T(A.eb[t][a][0]), s[0]);
    } else {
      p = vmul(T(-A.ea[t][a][0]), l[n - 1]);
      q = vmul(T(A.eb[t][a][0]), l[n - 1]);
    }
#pragma unroll
    for (int m = 1; m < h; ++m) vfma(p, T(A.ea[t][a][m]), d[m]);
#pragma unroll
    for (int m = 1; m < h; ++m) vfma(q, T(A.eb[t][a][m]), s[m]);
    if constexpr (n % 2 == 1) vfma(q, T(A.eb[t][a][h]), l[h]);
    emit(a, vadd(p, q));
    emit(n - 1 - a, vsub(p, q));
  }
  if constexpr (n % 2 == 1) {
    P o;
    if constexpr (TR) o = vmul(T(A.em[t][0]), d[0]);
    else o = vmul(T(-A.em[t][0]), l[n - 1]);
#pragma unroll
    for (int m = 1; m < h; ++m) vfma(o, T(A.em[t][m]), d[m]);
    emit(h, o);
  }
}

template <typename T, int N, int BB, int E, int FL>
__global__ void __launch_bounds__(VolTeam<N, E>::threads, vol_min_blocks<T, BB, N, E, FL>())
    hex_vol_kernel(const __grid_constant__ HexVolArgs<T> A) {
  using TM = VolTeam<N, E>;
  constexpr bool LEAN = (FL & VOL_LEAN) != 0, GSM = (FL & VOL_GSM) != 0, DB = (FL & VOL_DB) != 0;
  constexpr int n = TM::n, nl = TM::nl, gs = (nl + 3) / 4 * 4;
  constexpr int GPER = (E * nl + TM::threads - 1) / TM::threads;   // gather entries per thread
  using P = Pack<T, BB>;
  using SP = SPlanes<T, BB>;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr long long PL = (long long)E * nl * BB;                // one plane set of packs
  const SP Ub[2] = {{sm, E * nl}, {sm + (DB ? PL : 0), E * nl}};  // u, then F_z (LEAN) or R_x
  const SP G0 = {sm + (DB ? 2 : 1) * PL, E * nl};                 // grad^_x u, then F_x (then R_x: LEAN)
  const SP G1 = {sm + (DB ? 3 : 2) * PL, E * nl};                 // grad^_y u, then F_y, then R_y
  T* Gs = reinterpret_cast<T*>(smem_raw + vol_geo_off<T, BB, N, E, FL>());   // [E][6][gs] (GSM)
  const int t = threadIdx.x;
  const int el = t / TM::line, q = t - el * TM::line;
  const int e0 = blockIdx.x * E;
  const int e = e0 + el;
  const int ne_cta = min(E, A.ne - e0);
  const bool act = el < E && e < A.ne;
  const int qa = q % n, qb = q / n;          // the two line coordinates
  const int o = el * nl;                     // this element's entries in the shared arrays
  const int xb = o + n * qa + n * n * qb;    // x-line (b, c) = (qa, qb): entries xb + a
  const int yb = o + qa + n * n * qb;        // y-line (a, c) = (qa, qb): entries yb + n a
  const int zb = o + qa + n * qb;            // z-line (a, b) = (qa, qb): entries zb + n^2 c
  const T* gsm = GSM ? Gs + el * 6 * gs : (act ? A.G + 6LL * e * gs : A.G);
  const int nch = A.Bp / BB;
  // node ids of this thread's gather entries, reused by every chunk
  int nd[GPER];
#pragma unroll
  for (int g = 0; g < GPER; ++g) {
    const int i = t + g * TM::threads;
    nd[g] = i < ne_cta * nl ? A.conn[(long long)e0 * nl + i] : 0;
  }
  auto gather = [&](int ch, const SP& dst) {
#pragma unroll
    for (int g = 0; g < GPER; ++g) {
      const int i = t + g * TM::threads;
      if (i < ne_cta * nl) {
        const T* src = A.p + (long long)nd[g] * A.Bp + ch * BB;
#pragma unroll
        for (int pl = 0; pl < SP::NPL; ++pl)
          cp_async<(int)(SP::H * sizeof(T))>(dst.ptr(pl, i), src + pl * SP::H);
      }
    }
  };
  if constexpr (GSM) {
    constexpr int per16 = 16 / (int)sizeof(T);
    const T* gsrc = A.G + 6LL * e0 * gs;
    for (int i = t * per16; i < ne_cta * 6 * gs; i += blockDim.x * per16) cp_async16(Gs + i, gsrc + i);
  }
  if constexpr (DB) {
    gather(0, Ub[0]);
    cp_commit();
  }
  for (int ch = 0; ch < nch; ++ch) {
    const SP& U = Ub[DB ? (ch & 1) : 0];
    if constexpr (DB) {
      if (ch + 1 < nch) gather(ch + 1, Ub[(ch + 1) & 1]);
      cp_commit();
      cp_wait<1>();
    } else {
      gather(ch, U);
      cp_commit();
      cp_wait<0>();
    }
    __syncthreads();
    if (act) {
      // A: grad^_x u along the x-line, grad^_y u along the y-line
      {
        P l[n];
#pragma unroll
        for (int m = 0; m < n; ++m) l[m] = U.ld(xb + m);
        eo_line<T, BB, n, false>(A, l, [&](int a, const P& v) { G0.st(xb + a, v); });
      }
      {
        P l[n];
#pragma unroll
        for (int m = 0; m < n; ++m) l[m] = U.ld(yb + n * m);
        eo_line<T, BB, n, false>(A, l, [&](int a, const P& v) { G1.st(yb + n * a, v); });
      }
    }
    __syncthreads();
    P fz[LEAN ? 1 : n];
    if (act) {
      // B: z-line: grad^_z u, then F = G grad^ u at its nodes
      P l[n];
#pragma unroll
      for (int m = 0; m < n; ++m) l[m] = U.ld(zb + n * n * m);
      eo_line<T, BB, n, false>(A, l, [&](int c, const P& gz) {
        const int k = zb + n * n * c;
        const T* gp = gsm + (k - o);
        T G00, G11, G22, G01, G02, G12;
        if constexpr (GSM) {
          G00 = gp[0]; G11 = gp[gs]; G22 = gp[2 * gs]; G01 = gp[3 * gs]; G02 = gp[4 * gs]; G12 = gp[5 * gs];
        } else {
          G00 = __ldg(gp); G11 = __ldg(gp + gs); G22 = __ldg(gp + 2 * gs);
          G01 = __ldg(gp + 3 * gs); G02 = __ldg(gp + 4 * gs); G12 = __ldg(gp + 5 * gs);
        }
        const P gx = G0.ld(k), gy = G1.ld(k);
        P fx = vmul(G00, gx), fy = vmul(G01, gx), fzc = vmul(G02, gx);
        vfma(fx, G01, gy);
        vfma(fy, G11, gy);
        vfma(fzc, G12, gy);
        vfma(fx, G02, gz);
        vfma(fy, G12, gz);
        vfma(fzc, G22, gz);
        G0.st(k, fx);
        G1.st(k, fy);
        if constexpr (LEAN) U.st(k, fzc);   // the thread's own z-line entries, already read
        else fz[c] = fzc;
      });
    }
    __syncthreads();
    if (act) {
      // C: R_x = D^T F_x along the x-line (to U, or in place: LEAN); R_y = D^T F_y in place
      {
        P l[n];
#pragma unroll
        for (int m = 0; m < n; ++m) l[m] = G0.ld(xb + m);
        eo_line<T, BB, n, true>(A, l, [&](int a, const P& v) {
          if constexpr (LEAN) G0.st(xb + a, v);
          else U.st(xb + a, v);
        });
      }
      {
        P l[n];
#pragma unroll
        for (int m = 0; m < n; ++m) l[m] = G1.ld(yb + n * m);
        eo_line<T, BB, n, true>(A, l, [&](int a, const P& v) { G1.st(yb + n * a, v); });
      }
    }
    __syncthreads();
    if (act) {
      // D: z-line: r = R_x + R_y + D^T F_z -> the element's residual slots
      P* sout = reinterpret_cast<P*>(A.S + (A.slot_base + (long long)e * nl) * A.Bp) + ch;
      const SP& RX = LEAN ? G0 : U;
      auto out = [&](int c, const P& rz) {
        const int k = zb + n * n * c;
        sout[(long long)(k - o) * (A.Bp / BB)] = vadd(vadd(RX.ld(k), G1.ld(k)), rz);
      };
      if constexpr (LEAN) {
        P l[n];
#pragma unroll
        for (int m = 0; m < n; ++m) l[m] = U.ld(zb + n * n * m);
        eo_line<T, BB, n, true>(A, l, out);
      } else {
        eo_line<T, BB, n, true>(A, fz, out);
      }
    }
    __syncthreads();
  }
}

template <typename T, int N, int BB, int E, int FL>
cudaError_t vol_launch(const HexVolArgs<T>& a, cudaStream_t s) {
  using TM = VolTeam<N, E>;
  constexpr size_t sm = vol_smem<T, BB, N, E, FL>();
  if constexpr (sm > 227 * 1024) {
    // this shape does not fit one CTA at this order: the default form instead
    return vol_launch<T, N, BB, vol_e0<N>(), VOL_GSM | VOL_DB>(a, s);
  } else {
    if (sm > 48 * 1024) {
      const cudaError_t e =
          cudaFuncSetAttribute(hex_vol_kernel<T, N, BB, E, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    hex_vol_kernel<T, N, BB, E, FL><<<(a.ne + E - 1) / E, TM::threads, sm, s>>>(a);
    return cudaGetLastError();
  }
}

// Variant v of order N.  Batches not padded to the vector width V take the
// one-member kernel whatever v is; orders 1 and 2 take the default.  Per-
// kernel times on the distorted meshes (FP32 and FP64, 8 and 64 members)
// decided the set: the default (v 0) is fastest for order 4 at 64 FP32
// members, v 4 for order 6 there, v 3 (five order-6 elements per CTA, 4%
// idle lanes instead of 23%) for FP64, v 1, 2 and 4 for 8 FP32 members.
// Measured and left out: 8 FP32 members in the register form with five
// order-6 elements per CTA (one 220 KB CTA per SM), with the prefetch or with
// staged geometry: 1.3 and 3.2 ms slower than v 0 at 64 members.
template <typename T, int N>
cudaError_t vol_variant(const HexVolArgs<T>& a, int v, cudaStream_t s) {
  constexpr int V = vec_width<T>(), H = V / 2, E0 = vol_e0<N>(), E1 = vol_e1<N>();
  constexpr int L = VOL_LEAN, G = VOL_GSM, B2 = VOL_DB;
  if (a.Bp % V != 0) return vol_launch<T, N, 1, E0, G | B2>(a, s);
  if constexpr (N < 3) {
    return vol_launch<T, N, V, E0, G | B2>(a, s);
  } else {
    switch (v) {
      case 0: return vol_launch<T, N, V, E0, G | B2>(a, s);
      case 1: return vol_launch<T, N, H, E0, L | G | B2>(a, s);
      case 2: return vol_launch<T, N, H, E0, L | B2>(a, s);
      case 3: return vol_launch<T, N, H, E1, L | B2>(a, s);
      case 4: return vol_launch<T, N, V, E0, L>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

template <typename T>
cudaError_t launch_hex_vol_impl(const HexVolArgs<T>& a, int n, int variant, cudaStream_t s) {
  if (a.ne == 0 || a.Bp == 0) return cudaSuccess;
  if (variant < 0 || variant >= kHexVolVariants) return cudaErrorInvalidValue;
  switch (n - 1) {
    case 1: return vol_variant<T, 1>(a, variant, s);
    case 2: return vol_variant<T, 2>(a, variant, s);
    case 3: return vol_variant<T, 3>(a, variant, s);
    case 4: return vol_variant<T, 4>(a, variant, s);
    case 5: return vol_variant<T, 5>(a, variant, s);
    case 6: return vol_variant<T, 6>(a, variant, s);
    case 7: return vol_variant<T, 7>(a, variant, s);
    case 8: return vol_variant<T, 8>(a, variant, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hex
