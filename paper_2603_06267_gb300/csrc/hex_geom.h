// General hexahedra (trilinear elements, Sec. 3): geometry helpers used by the
// host setup and the CUDA kernels, and the parameter blocks of the kernels.
// Not part of the public ABI (include/dghex.h).
#pragma once

#include <cuda_runtime.h>

#ifdef __CUDACC__
#define HXD __host__ __device__ __forceinline__
#else
#define HXD inline
#endif

namespace hex {

constexpr int MAXN1 = 9;     // GLL nodes per direction (order <= 8)
constexpr int MAXQ = 9;      // Gauss points per direction on a fine face
constexpr int PDAT = 14;     // doubles per interface quadrature node
// per-point table of the face-collapsed interface kernel: l and l' along the
// two face axes of each side ([2 sides][2 axes][2][MAXN1]), then c+^2 a+
// (t0, t1, n), c-^2 a- (t0, t1, n), W, gamma
constexpr int kFaceTab = 8 * MAXN1 + 8;
// per-point table of the general interface kernel: l and l' along the three
// reference axes of each side ([2 sides][3 axes][2][MAXN1]), then a+ (3),
// a- (3), W, gamma
constexpr int kGenTab = 12 * MAXN1 + 8;

// Trilinear map of an element with corner vertices V (corner (i, j, k) at
// index i + 2 j + 4 k, reference corner (2i-1, 2j-1, 2k-1)): X(r) and
// J[i][d] = dX_i / dr_d.
HXD void tri_map(const double* V, const double* r, double* X, double J[3][3]) {
  double f[2][3];
  for (int d = 0; d < 3; ++d) {
    f[0][d] = 0.5 * (1.0 - r[d]);
    f[1][d] = 0.5 * (1.0 + r[d]);
  }
  for (int i = 0; i < 3; ++i) {
    X[i] = 0.0;
    J[i][0] = J[i][1] = J[i][2] = 0.0;
  }
  for (int c = 0; c < 8; ++c) {
    const int b0 = c & 1, b1 = (c >> 1) & 1, b2 = (c >> 2) & 1;
    const double s0 = b0 ? 0.5 : -0.5, s1 = b1 ? 0.5 : -0.5, s2 = b2 ? 0.5 : -0.5;
    const double n = f[b0][0] * f[b1][1] * f[b2][2];
    const double d0 = s0 * f[b1][1] * f[b2][2];
    const double d1 = f[b0][0] * s1 * f[b2][2];
    const double d2 = f[b0][0] * f[b1][1] * s2;
    for (int i = 0; i < 3; ++i) {
      const double v = V[3 * c + i];
      X[i] += n * v;
      J[i][0] += d0 * v;
      J[i][1] += d1 * v;
      J[i][2] += d2 * v;
    }
  }
}

// Inverse of a 3x3 matrix by its adjugate; returns the determinant.
HXD double inv3(const double J[3][3], double Ji[3][3]) {
  const double a00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double a01 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  const double a02 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  const double a10 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double a11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  const double a12 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  const double a20 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double a21 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  const double a22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * a00 + J[0][1] * a10 + J[0][2] * a20;
  const double s = 1.0 / det;
  Ji[0][0] = a00 * s; Ji[0][1] = a01 * s; Ji[0][2] = a02 * s;
  Ji[1][0] = a10 * s; Ji[1][1] = a11 * s; Ji[1][2] = a12 * s;
  Ji[2][0] = a20 * s; Ji[2][1] = a21 * s; Ji[2][2] = a22 * s;
  return det;
}

// Reference point of local face f = 2 axis + side at face coordinates (s, t)
// (the two other axes in increasing order).
HXD void face_ref(int f, double s, double t, double* r) {
  const int ax = f >> 1;
  const int t0 = ax == 0 ? 1 : 0, t1 = ax == 2 ? 1 : 2;
  r[ax] = (f & 1) ? 1.0 : -1.0;
  r[t0] = s;
  r[t1] = t;
}

// Outward unit normal and surface Jacobian |J| |J^-T e_axis| (Nanson) at a
// point of local face f, from the volume Jacobian there.
HXD double face_normal(int f, const double J[3][3], double* n) {
  double Ji[3][3];
  const double det = inv3(J, Ji);
  const int ax = f >> 1;
  const double g0 = Ji[ax][0], g1 = Ji[ax][1], g2 = Ji[ax][2];
  const double gn = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
  const double sg = (f & 1) ? 1.0 : -1.0;
  n[0] = sg * g0 / gn;
  n[1] = sg * g1 / gn;
  n[2] = sg * g2 / gn;
  return det * gn;
}

// Reference position of x in the element by Newton-Raphson on X(r) = x from
// the centre (Algorithm 3): at most maxit iterations, stop when the update is
// below 1e-15 in every component.  false when the iteration meets a singular
// Jacobian or leaves |r| < 16 (the point is far outside the element).
HXD bool newton_ref(const double* V, const double* x, double* r, int maxit = 50) {
  r[0] = r[1] = r[2] = 0.0;
  for (int it = 0; it < maxit; ++it) {
    double X[3], J[3][3], Ji[3][3];
    tri_map(V, r, X, J);
    const double det = inv3(J, Ji);
    if (!(det != 0.0) || !isfinite(det)) return false;
    double st[3], mx = 0.0;
    for (int i = 0; i < 3; ++i) {
      st[i] = Ji[i][0] * (X[0] - x[0]) + Ji[i][1] * (X[1] - x[1]) + Ji[i][2] * (X[2] - x[2]);
      r[i] -= st[i];
      mx = fmax(mx, fabs(st[i]));
    }
    if (!(fabs(r[0]) < 16.0 && fabs(r[1]) < 16.0 && fabs(r[2]) < 16.0)) return false;
    if (mx < 1e-15) break;
  }
  return true;
}

HXD bool inside_ref(const double* r) {
  return fabs(r[0]) <= 1.0 + 1e-10 && fabs(r[1]) <= 1.0 + 1e-10 && fabs(r[2]) <= 1.0 + 1e-10;
}

// Lagrange basis values and derivatives on GLL nodes xi[0..n-1] at t
// (product formula; derivative as the sum over the dropped factor).
HXD void lagrange(int n, const double* xi, double t, double* l, double* dl) {
  for (int a = 0; a < n; ++a) {
    double v = 1.0, d = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == a) continue;
      const double inv = 1.0 / (xi[a] - xi[m]);
      d = d * (t - xi[m]) * inv + v * inv;
      v *= (t - xi[m]) * inv;
    }
    l[a] = v;
    dl[a] = d;
  }
}

// ---------------------------------------------------------------------------
// Kernel parameter blocks
// ---------------------------------------------------------------------------
// Setup: geometric factors c^2 w_abc |J| J^-1 J^-T (6 symmetric entries, order
// 00 11 22 01 02 12) and w_abc |J| at every GLL node of every element.  The
// factors are stored [element][entry][gstride(n)] with the row padded to a
// multiple of 4 values, so every row starts on a 16-byte boundary.
HXD int gstride(int n) { return (n * n * n + 3) / 4 * 4; }
struct GeomArgs {
  const double* vert;   // [nv][3]
  const int* elem;      // [ne][8]
  int ne, n;            // elements, nodes per direction
  double xi[MAXN1], w[MAXN1];
  double c2;
  double* G64;          // [ne][6][gstride(n)]
  float* G32;
  double* Mloc;         // [ne][n^3] (volume slots of this domain)
  int* bad;             // count of nodes with |J| <= 0
};

// Setup: per face of a list, the data of Algorithm 3's filters and gamma_F.
struct FaceArgs {
  const double* vert;
  const int* elem;
  const int* faces;     // [nf][2] (element, local face)
  int nf, n;
  double xi[MAXN1], w[MAXN1];
  const double* Mloc;   // element volumes: sum of the element's Mloc
  double* out;          // [nf][8]: normal at the centre (3), stored vertex (3), diameter, h = |K| / |F|
};

// Setup: Algorithm 3 for every Gauss node of every fine face, then the
// per-node interface data.
struct MatchArgs {
  const double* vert_p; const int* elem_p; const int* ff; const double* fdat;   // fine side
  const double* vert_m; const int* elem_m; const int* cf; const double* cdat;   // coarse side
  int nff, ncf, q;
  double g[MAXQ], gw[MAXQ];
  double tol, eps;
  int* match;           // [nff q^2] coarse face index or -1
  double* refm;         // [nff q^2][3]
  // interface data (second kernel)
  double alpha_cbar2_n2;   // alpha cbar^2 max(N)^2
  double* pdat;         // [nff q^2][PDAT]: refp(3) refm(3) a+(3) a-(3) W gamma
};

// Step kernels keep every field batch-innermost: value (node j, member b) at
// j * Bp + b, Bp the batch padded to a multiple of the vector width (8 FP32 or
// 4 FP64 members = 32 bytes) when the batch is at least that wide.
//
// Step: element stiffness of one domain into its volume slots.
template <typename T>
struct HexVolArgs {
  const T* p; T* S;
  int Bp;                    // padded batch (row length of p and S)
  const int* conn;           // [ne][n^3] node ids
  const T* G;                // [ne][6][gstride(n)]
  long long slot_base;       // first volume slot of this domain
  int ne;
  // even-odd split of C = D ([0], D[i][j] = l_j'(xi_i)) and C = D^T ([1]),
  // h = n / 2: ea[a][m] = (C[a][m] - C[a][n-1-m]) / 2, eb[a][m] = (C[a][m] +
  // C[a][n-1-m]) / 2 (a, m < h), eb[a][h] = C[a][h], em[m] = C[h][m] (odd n)
  T ea[2][MAXN1 / 2][MAXN1 / 2];
  T eb[2][MAXN1 / 2][MAXN1 / 2 + 1];
  T em[2][MAXN1 / 2];
};

// Step: SIPG interface terms of one group (fine face, coarse element) into
// its slot block [n+^3 fine-element slots | n-^3 coarse-element slots].
template <typename T>
struct HexIfaceArgs {
  const T* p; T* S;
  int Bp;
  const int* conn_p; const int* conn_m;
  const int* g_fe; const int* g_ce;   // [ng] element ids
  const int* g_pt;                    // [ng+1] CSR into pt_idx
  const int* pt_idx;                  // interface node ids (rows of pdat)
  const long long* g_slot;            // [ng] first slot of the group's block
  const int* g_face;                  // [ng][2] local face of K+ and of K- (face kernel)
  const double* pdat;
  double xip[MAXN1], xim[MAXN1];
  T Dp[MAXN1][MAXN1], Dm[MAXN1][MAXN1];   // derivative matrices of the two orders (face kernel)
  int np, nm;                         // GLL nodes per direction, fine / coarse
  double c2p, c2m;
  int ng, max_pts;
  int onface;                         // every Gauss node lies on one face of each side's element
  const T* ftab;                      // [g_pt[ng]][kFaceTab] per-point tables of the face kernel
  const T* gtab;                      // [g_pt[ng]][kGenTab] per-point tables of the general kernel
};

// Step: residual assembly (sum of a node's slots in ascending slot order)
// and the leapfrog update v += cv (damp v + M^-1 r), p_out = p_in + cp v.
template <typename T>
struct HexUpdateArgs {
  const T* p_in; T* p_out; T* v; const T* S;
  int Bp;
  const int* node_ptr; const int* node_slot;
  const T* Minv;
  const T* damp;             // C_jj / M_jj + alpha_j (absorbing faces, layers), or NULL
  // perfectly matched layers (or NULL): v += cv (beta p + gamma psi_int) with
  // psi_int = psi + hpsi p_in, then psi += dpsi p_in
  const T* beta; const T* gamma; T* psi;
  T hpsi, dpsi;
  long long ndof;
  T cv, cp;
};

// Step: one layer element per CTA (one node per thread): Phi^{n+1/2} ->
// Phi^{n+3/2} by Crank-Nicolson and the residual G (Phi^{n+1/2} + Phi^{n+3/2})/2
// into the element's layer slots.
template <typename T>
struct HexPmlArgs {
  const T* p;                // p^{n+1}
  const T* psi;              // psi^{n+1/2}
  T* phi;                    // [npml][3][n^3][Bp]
  T* S;
  int Bp;
  const int* elem;           // [npml] element ids
  const int* conn;           // [ne][n^3]
  const T* geo;              // [npml][10][n^3]: J^-1 (row-major), w |J|
  const T* zeta;             // [3][ndof]
  long long ndof;
  long long slot_base;       // first layer slot of this domain (element-major)
  int npml;
  T c2, dt;
  T D[MAXN1][MAXN1];
};

// Step tail: PMUT forcing slots kappa sum_m q''_km B_jm of every footprint
// entry, receiver samples of p^{n+1}, then the step counter advances.
template <typename T>
struct HexTailArgs {
  int nnz, M, K, B, Bp;
  const int* ent_k; const double* Bm; const double* qdd;
  double kappa;
  T* S; long long fslot;
  int R, rstride;
  const double* rw; const long long* roff; const int* rnn;   // roff: node ids
  const T* p;
  double* traces; long long tbs, trs;
  int n; int* step; unsigned* done;
  int fblocks;
};

cudaError_t launch_geom(const GeomArgs& a, cudaStream_t s);
cudaError_t launch_mass(const double* Mloc, const int* node_ptr, const int* node_slot, long long nvol, long long ndof,
                        double* Minv64, float* Minv32, double* M, cudaStream_t s);
cudaError_t launch_faces(const FaceArgs& a, cudaStream_t s);
cudaError_t launch_match(const MatchArgs& a, cudaStream_t s);
cudaError_t launch_ipoints(const MatchArgs& a, cudaStream_t s);
cudaError_t launch_norm2(const double* x, long long n, double* out, cudaStream_t s);
cudaError_t launch_energy(const double* M, const double* v, const double* p, const double* w, long long ndof, int B,
                          int Bp, double* e, cudaStream_t s);
cudaError_t launch_scale(double* dst, const double* src, const double* norm2, long long n, cudaStream_t s);
template <typename T> cudaError_t launch_hex_pml(const HexPmlArgs<T>& a, int n, cudaStream_t s);
// element stiffness, launch variant 0 .. kHexVolVariants - 1 (same results)
constexpr int kHexVolVariants = 5;
template <typename T> cudaError_t launch_hex_vol(const HexVolArgs<T>& a, int n, int variant, cudaStream_t s);
template <typename T> cudaError_t launch_hex_iface(const HexIfaceArgs<T>& a, cudaStream_t s);
// setup: the face kernel's per-point tables in the working precision (once per precision)
template <typename T> cudaError_t launch_hex_iface_table(const HexIfaceArgs<T>& a, T* tab, cudaStream_t s);
template <typename T> cudaError_t launch_hex_iface_gtable(const HexIfaceArgs<T>& a, T* tab, cudaStream_t s);
template <typename T> cudaError_t launch_hex_update(const HexUpdateArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_hex_tail(const HexTailArgs<T>& a, cudaStream_t s);

}  // namespace hex
