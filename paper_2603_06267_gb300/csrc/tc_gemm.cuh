// BF16 GEMM on the fifth-generation tensor cores (tcgen05), FP32 accumulation
// in tensor memory, for the dense layers of the learned surrogate.
//
//     C[m][n] = sum_k A[m][k] B[n][k]        (A [M][K], B [N][K], both K-contiguous)
//
// One CTA computes a 128 x BN tile of C.  Thread 0 streams 128 x 64 tiles of A
// (rows of a matrix, or time-shifted rows of a [batch][time][channel] array
// for the transposed convolutions) and BN x 64 tiles of B into a ring of
// shared-memory stages with TMA
// (cp.async.bulk.tensor, 128-byte swizzle); thread 32 issues tcgen05.mma
// (kind::f16, BF16 inputs, M = 128, N = BN, K = 16 per instruction) into a
// 128-lane x BN-column FP32 accumulator in tensor memory, and releases each
// stage through tcgen05.commit on the stage's "empty" mbarrier; after the last
// k-tile a final commit signals the epilogue, in which every warp reads its 32
// accumulator lanes (tcgen05.ld 32x32b) and applies bias, GELU and the BF16
// copy.  Every mbarrier wait is bounded; a wait that gives up sets *err and
// the kernel finishes without further tensor-memory reads.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tcg {

constexpr int BM = 128;   // rows of a C tile (= accumulator lanes)
constexpr int BK = 64;    // k-extent of a stage: one 128-byte swizzle row of BF16
constexpr int THREADS = 128;

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
// gives up after about a second of SM clocks
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// Where the 128 x 64 A tile of k-tile kt and row tile mt comes from.
// DenseA: rows mt*128 .. of a 2-D [M][K] matrix.
struct DenseA {
  __device__ __forceinline__ void operator()(void* dst, const CUtensorMap* map, uint64_t* bar, int kt, int mt) const {
    tma_load_2d(dst, map, bar, kt * BK, mt * BM);
  }
};
// ShiftA: the rows of a 3-D [B][T][C] array taken as (b, t) pairs, t fastest
// (T divides 128 or 128 divides T); the first kh k-tiles read channels
// 64 kt .. at time t + sh0, the others channels 64 (kt - kh) .. at time
// t + sh1.  Rows shifted past either end of the time axis read zeros.
struct ShiftA {
  int kh, T, sh0, sh1;
  __device__ __forceinline__ void operator()(void* dst, const CUtensorMap* map, uint64_t* bar, int kt, int mt) const {
    const bool second = kt >= kh;
    const int c0 = (second ? kt - kh : kt) * BK;
    const int sh = second ? sh1 : sh0;
    const int r0 = mt * BM;
    tma_load_3d(dst, map, bar, c0, (r0 % T) + sh, r0 / T);
  }
};

// SegA: rows (b, t) of a 4-D [P][B][T][C] array, t fastest (T divides 128
// or 128 divides T); the K axis is nseg segments of C channels each, segment
// g read at time t + sh[g] from plane pl[g].  Rows shifted past either end of
// the time axis read zeros.
struct SegA {
  int kseg, T;
  int sh[4], pl[4];
  __device__ __forceinline__ void operator()(void* dst, const CUtensorMap* map, uint64_t* bar, int kt, int mt) const {
    const int g = kt / kseg;
    const int c0 = (kt - g * kseg) * BK;
    const int r0 = mt * BM;
    tma_load_4d(dst, map, bar, c0, (r0 % T) + sh[g], r0 / T, pl[g]);
  }
};

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row (1024-byte) swizzle atoms
// stacked along M/N.  Start address >> 4 (bits 0-13); leading byte offset
// (bits 16-29, not used by swizzled K-major layouts, set to 16 bytes); stride
// byte offset between 8-row groups, 1024 bytes (bits 32-45); descriptor
// version 1 (bits 46-47); base offset 0 (the atoms start 1024-byte aligned);
// layout type 2 = 128-byte swizzle (bits 61-63).  A k-slice of 16 elements
// (32 bytes) inside the swizzle row is addressed by advancing the start.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), BF16 A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16
// = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on bar once every tcgen05.mma this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN, int STAGES>
struct Geo {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int BAR_OFF = STAGES * STAGE;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;   // barriers, TMEM slot, 1024-byte alignment slack
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "stages must keep 1024-byte alignment");
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "BN: a power of two in [32, 256]");
  static_assert(SMEM <= 227 * 1024, "stages exceed shared memory");
};

// An epilogue functor with `static constexpr bool paired = true` receives the
// accumulator columns c and c + BN/2 of a row together.
template <typename E, typename = void> struct PairedEpilogue { static constexpr bool value = false; };
template <typename E> struct PairedEpilogue<E, decltype(void(E::paired))> { static constexpr bool value = E::paired; };

// Epilogue of the surrogate's dense layers: + bias[n]; FP32 copy to C (ldc);
// BF16 copy of gelu(.) (act = 1) or of the value (act = 0) to Cb (ldcb).
struct Epi {
  const float* bias;
  float* C; int ldc;
  __nv_bfloat16* Cb; int ldcb; int act;
};

template <int BN, int STAGES, typename EpiFn, typename ALoad = DenseA>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int K,
                EpiFn epi, int* err, ALoad aload) {
  using G = Geo<BN, STAGES>;
  extern __shared__ unsigned char raw[];
  // 1024-byte aligned base of the stages (128-byte swizzle atoms)
  const uint32_t raw_s = smem_u32(raw);
  unsigned char* base = raw + ((1024u - (raw_s & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + G::BAR_OFF);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // split K: CTA z of gridDim.z takes k-tiles kt0 .. kt0 + KT - 1 (the
  // epilogue sees blockIdx.z and writes that part's partial sum)
  const int KT = K / BK / gridDim.z;
  const int kt0 = blockIdx.z * KT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA fills of the stages
    int issued = 0;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((kt / STAGES) - 1) & 1))) {
        atomicExch(err, 1);
        break;
      }
      unsigned char* st = base + s * G::STAGE;
      mbar_expect_tx(&full[s], (uint32_t)G::STAGE);
      aload(st, &tmA, &full[s], kt0 + kt, blockIdx.y);
      tma_load_2d(st + G::A_BYTES, &tmB, &full[s], (kt0 + kt) * BK, n0);
      issued = kt + 1;
    }
    // every fill issued has landed before the CTA can leave
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
      (void)mbar_wait(&full[kt % STAGES], (uint32_t)((kt / STAGES) & 1));
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t ID = idesc_bf16(BM, BN);
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)((kt / STAGES) & 1))) {
        atomicExch(err, 1);
        break;
      }
      fence_after_sync();
      const uint32_t a = smem_u32(base + s * G::STAGE), b = a + G::A_BYTES;
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        mma_bf16(tmem, sw128_desc(a + 32 * k), sw128_desc(b + 32 * k), ID, (kt | k) != 0 ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  // epilogue: warp w holds accumulator lanes (rows) 32w .. 32w + 31
  const bool ready = mbar_wait(done, 0);
  if (!ready) atomicExch(err, 1);
  fence_after_sync();
  if (ready && *reinterpret_cast<volatile int*>(err) == 0) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    if constexpr (PairedEpilogue<EpiFn>::value) {
      // the tile's two column halves belong together (column c and c + BN/2)
#pragma unroll 1
      for (int c0 = 0; c0 < BN / 2; c0 += 32) {
        uint32_t r[32], q[32];
        tmem_ld32(tl + (uint32_t)c0, r);
        tmem_ld32(tl + (uint32_t)(c0 + BN / 2), q);
        if (row < M) epi(row, n0 + c0, r, q);
      }
    } else {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tl + (uint32_t)c0, r);
        if (row < M) epi(row, n0 + c0, r);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
  }
}

}  // namespace tcg
