// Fused volume step of one box: M^-1 (f - K p) with the sum-factorised GLL
// stiffness of eq. (Wf_2), the PMUT forcing of eq. (f_i) on the z-min plane,
// the SIPG interface residual of the interface element layer, and the
// leapfrog form of the Newmark gamma=1/2, beta=0 corrector/predictor of
// Algorithm 1:  v <- v + dtv * a,  p_out <- p_in + dtp * v.
//
// Layout: one lattice of GLL nodes per box, x fastest, padded row pitch.
// Work decomposition: a CTA owns an element-aligned x-y tile of TXE element
// columns x (TYE*N) rows and marches over a chunk of element layers in z.
// Each thread owns the N nodes of one element along x in one row.  For each
// layer the N+1 planes of the layer are staged in shared memory with a halo
// of one element on the low x/y side and one node on the high side (vertex
// rows need the neighbouring element, interior rows only their own); the
// z-direction coupling to the layer below is carried in registers as a
// partial sum, so no z halo is loaded.
#include "internal.h"

namespace {

template <typename T, int N>
__device__ __forceinline__ T face_gather(const T* __restrict__ R, int i, int j, int ne0, int ne1) {
  // Sum of the per-face (unassembled) residual entries that touch node (i, j)
  // of the face lattice, in a fixed order (deterministic).
  int fx = i / N, ax = i - fx * N;
  int fy = j / N, ay = j - fy * N;
  if (fx == ne0) { fx = ne0 - 1; ax = N; }
  if (fy == ne1) { fy = ne1 - 1; ay = N; }
  constexpr int F = (N + 1) * (N + 1);
  T s = R[(long long)(fy * ne0 + fx) * F + ay * (N + 1) + ax];
  if (ax == 0 && fx > 0) s += R[(long long)(fy * ne0 + fx - 1) * F + ay * (N + 1) + N];
  if (ay == 0 && fy > 0) s += R[(long long)((fy - 1) * ne0 + fx) * F + N * (N + 1) + ax];
  if (ax == 0 && fx > 0 && ay == 0 && fy > 0)
    s += R[(long long)((fy - 1) * ne0 + fx - 1) * F + N * (N + 1) + N];
  return s;
}

template <typename T, int N, int TXE, int TYE>
struct VolTile {
  static constexpr int TYR = TYE * N;              // owned rows
  static constexpr int COLS = TXE * N + N + 1;     // staged columns
  static constexpr int CP = (COLS + 3) & ~3;       // smem row pitch
  static constexpr int ROWS = TYR + N + 1;         // staged rows
  static constexpr int PLANE = ROWS * CP;
  static constexpr int NT = TXE * TYR;             // threads
  static constexpr size_t SMEM = sizeof(T) * (size_t)(N + 1) * PLANE;
  // the staging loop hands whole rows to whole warps
  static_assert(NT % 32 == 0, "CTA must be a whole number of warps");
  static_assert(SMEM <= 227 * 1024, "tile exceeds shared memory");
};

// Rare per-node terms: PMUT forcing f (eq. f_i) on the z-min plane and the
// interface residual of the interface element layer, both times M^-1.
template <typename T, int N>
__device__ __noinline__ T node_extras(const VolArgs<T, N>& A, int i, int j, int k, int b, T minv_t, double minv, T ra,
                                      T rb, bool iface_here) {
  T acc = T(0);
  if (A.has_pmut && k == 0) {
    double f = 0.0;
    const int e0 = A.node_ptr[j * A.L0 + i], e1 = A.node_ptr[j * A.L0 + i + 1];
    for (int e = e0; e < e1; ++e) {
      const int ent = A.node_ent[e];
      const double* qd = A.qdd + ((long long)b * A.K + A.ent_pmut[ent]) * A.M;
      const double* Bv = A.Bm + (long long)ent * A.M;
      for (int m = 0; m < A.M; ++m) f += qd[m] * Bv[m];
    }
    acc += T(-A.kappa * f * minv);
  }
  if (iface_here) {
    const int idx = k - A.iface_k0;
    if (idx >= 0 && idx <= N) {
      T r = A.dI[idx] * rb;
      if (idx == (A.iface_top ? N : 0)) r += ra;
      acc -= r * minv_t;
    }
  }
  return acc;
}

// x and y stencils of node (i = ex*N + a, j) in plane P, plus the update.
template <typename T, int N, int CP>
__device__ __forceinline__ void node_update(const VolArgs<T, N>& A, const T* __restrict__ P, int a, int i, int j, int k,
                                            int b, int r0, int cb, bool xl, bool xr, T xiw, bool yvert, bool yl,
                                            bool yr, T yiw, int yb, const T (&cyi)[N + 1], T iw_y, T zs, T iw_z,
                                            bool extras_layer, T ra, T rb, bool iface_here, T* __restrict__ pout,
                                            T* __restrict__ vv) {
  const int col = cb + a;
  T xs, iw_x;
  if (a == 0) {
    T l = T(0), r = T(0);
    if (xl) {
#pragma unroll
      for (int q = 0; q <= N; ++q) l += A.lx[q] * P[r0 * CP + cb - N + q];
    }
    if (xr) {
#pragma unroll
      for (int q = 0; q <= N; ++q) r += A.rx[q] * P[r0 * CP + cb + q];
    }
    xs = (l + r) * xiw;
    iw_x = xiw;
  } else {
    T s = T(0);
#pragma unroll
    for (int q = 0; q <= N; ++q) s += A.cx[a][q] * P[r0 * CP + cb + q];
    xs = s;
    iw_x = A.iwa[a];
  }
  T ys;
  if (yvert) {
    T l = T(0), r = T(0);
    if (yl) {
#pragma unroll
      for (int q = 0; q <= N; ++q) l += A.ly[q] * P[(r0 - N + q) * CP + col];
    }
    if (yr) {
#pragma unroll
      for (int q = 0; q <= N; ++q) r += A.ry[q] * P[(r0 + q) * CP + col];
    }
    ys = (l + r) * yiw;
  } else {
    T s = T(0);
#pragma unroll
    for (int q = 0; q <= N; ++q) s += cyi[q] * P[(r0 - yb + q) * CP + col];
    ys = s;
  }
  T acc = -(xs + ys + zs);
  if (extras_layer) {
    const T minv_t = T(A.minv_scale) * iw_x * iw_y * iw_z;
    const double minv = A.minv_scale * (double)iw_x * (double)iw_y * (double)iw_z;
    acc += node_extras<T, N>(A, i, j, k, b, minv_t, minv, ra, rb, iface_here);
  }
  const long long g = (long long)k * A.pz + (long long)j * A.py + i;
  const T vn = vv[g] + A.dtv * acc;
  vv[g] = vn;
  pout[g] = P[r0 * CP + col] + A.dtp * vn;
}

template <typename T, int N, int TXE, int TYE>
__global__ void __launch_bounds__(TXE * TYE * N)
vol_kernel(const __grid_constant__ VolArgs<T, N> A) {
  using Tile = VolTile<T, N, TXE, TYE>;
  constexpr int TYR = Tile::TYR, COLS = Tile::COLS, CP = Tile::CP, ROWS = Tile::ROWS;
  constexpr int PLANE = Tile::PLANE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TXE + tx;
  const int ex0 = blockIdx.x * TXE;
  const int x0 = ex0 * N;
  const int y0 = blockIdx.y * TYR;
  const int chunk = blockIdx.z % A.nchunks;
  const int b = blockIdx.z / A.nchunks;
  const int ez0 = chunk * A.layers_per_cta;
  const int ez1 = min(ez0 + A.layers_per_cta, A.ne2);
  const T* __restrict__ pin = A.p_in + (long long)b * A.bstride;
  T* __restrict__ pout = A.p_out + (long long)b * A.bstride;
  T* __restrict__ vv = A.v + (long long)b * A.bstride;

  const int ex = ex0 + tx;          // element column of this thread (ex == ne0: lone last vertex)
  const int j = y0 + ty;            // lattice row
  const bool row_ok = j < A.L1;
  const int ey = j / N;
  const int yb = j - ey * N;        // local row index in its element
  const bool yvert = (yb == 0);
  const bool yl = ey > 0, yr = ey < A.ne1;
  const T yiw = (yl && yr) ? A.iwv : A.iwb;
  T cyi[N + 1];
#pragma unroll
  for (int q = 0; q <= N; ++q) cyi[q] = yvert ? T(0) : A.cy[yb][q];
  const T iw_y = yvert ? yiw : A.iwa[yb];
  const bool xl = ex > 0, xr = ex < A.ne0;
  const T xiw = (xl && xr) ? A.iwv : A.iwb;

  // smem coordinates of this thread's first node (node ex*N)
  const int r0 = ty + N;            // staged row of row j
  const int cb = N + tx * N;        // staged column of node ex*N

  // interface residual of this column (gathered once)
  T ra[N], rb[N];
  const bool iface_here = A.iface_k0 >= 0 && A.iface_k0 <= ez1 * N && A.iface_k0 + N >= ez0 * N;
#pragma unroll
  for (int a = 0; a < N; ++a) { ra[a] = T(0); rb[a] = T(0); }
  if (iface_here && row_ok) {
    const T* Rab = A.Ra + (long long)b * (A.ne0 * A.ne1) * (N + 1) * (N + 1);
    const T* Rbb = A.Rb + (long long)b * (A.ne0 * A.ne1) * (N + 1) * (N + 1);
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int i = ex * N + a;
      if (i < A.L0) {
        ra[a] = face_gather<T, N>(Rab, i, j, A.ne0, A.ne1);
        rb[a] = face_gather<T, N>(Rbb, i, j, A.ne0, A.ne1);
      }
    }
  }

  // z carry: sum_b lz[b] p[(ez-1)N + b] of each owned node
  T carry[N];
#pragma unroll
  for (int a = 0; a < N; ++a) carry[a] = T(0);
  if (ez0 > 0 && row_ok) {
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int i = ex * N + a;
      if (i < A.L0) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q <= N; ++q)
          s += A.lz[q] * pin[(long long)((ez0 - 1) * N + q) * A.pz + (long long)j * A.py + i];
        carry[a] = s;
      }
    }
  }

  const int warp = tid >> 5, lane = tid & 31;
  constexpr int NWARP = (Tile::NT + 31) / 32;

  for (int ez = ez0; ez < ez1; ++ez) {
    __syncthreads();
    // stage planes ez*N .. ez*N+N, rows y0-N .. y0+TYR, columns x0-N .. x0+TXE*N
    for (int rr = warp; rr < (N + 1) * ROWS; rr += NWARP) {
      const int c = rr / ROWS, r = rr - c * ROWS;
      const int gk = ez * N + c, gj = y0 - N + r;
      const bool ok = gj >= 0 && gj < A.L1;
      const T* src = pin + (long long)gk * A.pz + (long long)gj * A.py;
      T* dst = S + c * PLANE + r * CP;
      for (int col = lane; col < COLS; col += 32) {
        const int gi = x0 - N + col;
        dst[col] = (ok && gi >= 0 && gi < A.L0) ? src[gi] : T(0);
      }
    }
    __syncthreads();
    if (!row_ok) continue;
    const bool extras_layer = (A.has_pmut && ez == 0) ||
                              (iface_here && A.iface_k0 <= ez * N + N && A.iface_k0 + N >= ez * N);
    // vertex plane c = 0: left part carried from the layer below
    {
      const int k = ez * N;
      const T iw_z = (ez > 0) ? A.iwv : A.iwb;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const int i = ex * N + a;
        if (i < A.L0) {
          T zr = T(0);
#pragma unroll
          for (int q = 0; q <= N; ++q) zr += A.rz[q] * S[q * PLANE + r0 * CP + cb + a];
          const T zs = (carry[a] + zr) * iw_z;
          node_update<T, N, CP>(A, S, a, i, j, k, b, r0, cb, xl, xr, xiw, yvert, yl, yr, yiw, yb, cyi, iw_y, zs, iw_z,
                                extras_layer, ra[a], rb[a], iface_here, pout, vv);
        }
      }
    }
    // interior planes c = 1 .. N-1
#pragma unroll 1
    for (int c = 1; c < N; ++c) {
      const int k = ez * N + c;
      const T iw_z = A.iwa[c];
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const int i = ex * N + a;
        if (i < A.L0) {
          T zs = T(0);
#pragma unroll
          for (int q = 0; q <= N; ++q) zs += A.cz[c][q] * S[q * PLANE + r0 * CP + cb + a];
          node_update<T, N, CP>(A, S + c * PLANE, a, i, j, k, b, r0, cb, xl, xr, xiw, yvert, yl, yr, yiw, yb, cyi, iw_y,
                                zs, iw_z, extras_layer, ra[a], rb[a], iface_here, pout, vv);
        }
      }
    }
    // carry for the vertex plane (ez+1)*N
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q <= N; ++q) s += A.lz[q] * S[q * PLANE + r0 * CP + cb + a];
      carry[a] = s;
    }
    // top boundary plane of the box (only the layer below exists)
    if (ez == A.ne2 - 1) {
      const int k = A.ne2 * N;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const int i = ex * N + a;
        if (i < A.L0) {
          node_update<T, N, CP>(A, S + N * PLANE, a, i, j, k, b, r0, cb, xl, xr, xiw, yvert, yl, yr, yiw, yb, cyi, iw_y,
                                carry[a] * A.iwb, A.iwb, extras_layer, ra[a], rb[a], iface_here, pout, vv);
        }
      }
    }
  }
}

template <typename T, int N>
VolArgs<T, N> make_args(const VolSpec& s) {
  VolArgs<T, N> a;
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
  a.iwv = T(s.iwv); a.iwb = T(s.iwb);
  a.minv_scale = s.minv_scale;
  a.has_pmut = s.has_pmut;
  a.node_ptr = s.node_ptr; a.node_ent = s.node_ent; a.ent_pmut = s.ent_pmut;
  a.Bm = s.Bm; a.qdd = s.qdd; a.K = s.K; a.M = s.M; a.kappa = s.kappa;
  a.iface_k0 = s.iface_k0; a.iface_top = s.iface_top;
  a.Ra = static_cast<const T*>(s.Ra); a.Rb = static_cast<const T*>(s.Rb);
  return a;
}

template <typename T, int N>
struct TileChoice {
  // element columns per CTA along x and element rows along y
  static constexpr int TXE = (N <= 4) ? 32 : 16;
  static constexpr int TYE = (N <= 2) ? 16 / N : ((N <= 4) ? 4 : (N <= 7 ? 2 : 1));
};

template <typename T, int N>
cudaError_t launch_n(const VolSpec& s, int batch, cudaStream_t st) {
  constexpr int TXE = TileChoice<T, N>::TXE, TYE = TileChoice<T, N>::TYE;
  using Tile = VolTile<T, N, TXE, TYE>;
  VolArgs<T, N> a = make_args<T, N>(s);
  int layers = s.layers_per_cta;
  const int gx = (s.L[0] + TXE * N - 1) / (TXE * N);
  const int gy = (s.L[1] + Tile::TYR - 1) / Tile::TYR;
  if (layers <= 0) {
    // enough CTAs to cover the GPU several times over
    const long long cols = (long long)gx * gy * batch;
    layers = s.ne[2];
    while (layers > 1 && cols * ((s.ne[2] + layers - 1) / layers) < 4 * 152) layers = (layers + 1) / 2;
  }
  a.layers_per_cta = layers;
  a.nchunks = (s.ne[2] + layers - 1) / layers;
  auto kern = vol_kernel<T, N, TXE, TYE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(gx, gy, a.nchunks * batch);
  dim3 block(TXE, Tile::TYR, 1);
  kern<<<grid, block, Tile::SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_vol(const VolSpec& s, int batch, cudaStream_t st) {
  switch (s.N) {
    case 1: return launch_n<T, 1>(s, batch, st);
    case 2: return launch_n<T, 2>(s, batch, st);
    case 3: return launch_n<T, 3>(s, batch, st);
    case 4: return launch_n<T, 4>(s, batch, st);
    case 5: return launch_n<T, 5>(s, batch, st);
    case 6: return launch_n<T, 6>(s, batch, st);
    case 7: return launch_n<T, 7>(s, batch, st);
    case 8: return launch_n<T, 8>(s, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_vol<float>(const VolSpec&, int, cudaStream_t);
template cudaError_t launch_vol<double>(const VolSpec&, int, cudaStream_t);
