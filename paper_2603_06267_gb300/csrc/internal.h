// Internal parameter blocks shared by the host setup (api.cu) and the CUDA
// kernels (vol.cu, small.cu).  Not part of the public ABI (include/dgsem.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#define DG_MAXN 8          // highest GLL order supported
#define DG_MAXM 16         // modes per PMUT
#define DG_MAXQ 12         // Gauss points per direction on a fine face

// ---------------------------------------------------------------------------
// Volume step of one box (fused: stiffness apply + forcing + interface
// residual + lumped-mass update + leapfrog corrector/predictor).
//
// For an affine box of equal elements the GLL stiffness of eq. (Wf_2)
// factorises as K = c^2 |J| sum_d (2/h_d)^2 (A (x) W (x) W)_d with the 1D
// GLL stiffness A = D^T W D and the 1D GLL weights W; the lumped mass is
// |J| W (x) W (x) W.  M^-1 K p is therefore a sum of three assembled 1D
// stencils along lattice lines, each row scaled by the inverse assembled
// 1D weight.  The coefficient blocks below hold those rows.
// ---------------------------------------------------------------------------
template <typename T, int N>
struct VolArgs {
  CUtensorMap tmap;    // 4D (x, y, z, batch) tiled view of p_in for the TMA staging loads
  CUtensorMap tmap_v;  // same view of v (used when v is staged too; also the v store box)
  CUtensorMap tmap_pst;  // view of p_out with the v box (TMA-store tile variants)
  int* err;            // device status word: set to 1 if a bounded wait gives up
  int* step;           // if not NULL, block (0,0,0) advances the run's step counter
  const T* p_in;       // p^{n+1}: stencil source
  T* p_out;            // p^{n+2} = p^{n+1} + dtp * v_new
  T* v;                // v^{n+1/2} -> v^{n+3/2} = v + dtv * a
  long long bstride;   // elements between batch members
  int L0, L1, L2;      // lattice nodes per axis (nelem*N + 1)
  int ne0, ne1, ne2;   // elements per axis
  int py;              // row pitch (elements)
  long long pz;        // plane pitch (elements)
  int layers_per_cta;  // element layers per CTA (z chunk)
  int nchunks;         // z chunks per batch member
  T dtv, dtp;
  // interior rows a = 1..N-1 of direction d: s_d A[a][b] / w_a  (s_d = c^2 (2/h_d)^2)
  T cx[N + 1][N + 1];
  T cy[N + 1][N + 1];
  T cz[N + 1][N + 1];
  // vertex rows: left element part s_d A[N][b], right element part s_d A[0][b]
  T lx[N + 1], rx[N + 1], ly[N + 1], ry[N + 1], lz[N + 1], rz[N + 1];
  T iwv;               // 1 / (w_0 + w_N): vertex shared by two elements
  T iwb;               // 1 / w_0: vertex on the box boundary
  T iwa[N + 1];        // 1 / w_a for interior rows (a = 1..N-1)
  double minv_scale;   // 8 / (hx hy hz)
  // PMUT forcing f on the z-min plane (primary box only), assembled per face
  // node for this step: fpm[b][j][i] = -kappa sum_entries sum_m q'' B  (eq. f_i)
  int has_pmut;
  const T* fpm;
  // interface residual (SIPG terms of eq. Wf_2), assembled per face node:
  // the nodes of the interface element layer get -(d_c gb + [c = top] ga)
  int iface_k0;            // first lattice plane of the interface element layer, -1: none
  int iface_top;           // 1: the value term sits on plane k0+N (primary), 0: on k0 (secondary)
  const T* ga;             // [B][L1][py]: sum over faces of sum_q l_a l_b alpha_q
  const T* gb;             // [B][L1][py]: sum over faces of sum_q l_a l_b beta_q
  long long gbs;           // batch stride of fpm / ga / gb
  T dI[N + 1];             // d_c = (2/h_z) l_c'(face)
  // absorbing sides (eq. Wf_4): sigma = C_ii / M_ii = c (2/h_d) / w_0 per box
  // side (x-, x+, y-, y+, z-, z+), 0 = rigid; a -= sigma v on those nodes
  T abc[6];
  int has_abc;
  // perfectly matched layer (eq. full_problem rows 1-3): on the nodes of the
  // layer's elements a -= beta p + alpha v + gamma psi^{n+1} + M^-1 (G Phi)
  // and psi^{n+3/2} = psi^{n+1/2} + dt p^{n+1}
  int has_pml, pml_init;           // pml_init: initial half step (no psi, no G Phi)
  const T* zeta[3];                // per-axis profiles zeta_d[L_d]
  T* psi;                          // psi at half steps, lattice layout
  const T* rpml;                   // [B][npml][(N+1)^3] G Phi^{n+1} per layer element
  const int* pml_slot;             // [ne2][ne1][ne0] slot in rpml, -1 outside the layer
  long long rpml_bs;               // batch stride of rpml
  int pml_lo[3], pml_hi[3];        // layer elements per axis at the low / high side
  // FP32 tables for packed f32x2 arithmetic: x rows with their taps in pairs
  // (q = 2k, 2k+1), y and z coefficients repeated in both lanes
  float2 cxq[N + 1][(N + 1) / 2];
  float2 lxq[(N + 1) / 2], rxq[(N + 1) / 2];
  float2 ly2[N + 1], ry2[N + 1], lz2[N + 1], rz2[N + 1];
  float2 cz2[N + 1][N + 1];
};

// ---------------------------------------------------------------------------
// Interface fluxes on Gamma_I (Sec. 5): one CTA per listed coarse face.
// ---------------------------------------------------------------------------
template <typename T>
struct IfaceArgs {
  const T* pp;  const T* ps;       // p^{n+1} of the primary / secondary box
  long long bsp, bss;              // batch strides
  int pyp; long long pzp;
  int pys; long long pzs;
  int Np, Ns, kp0;                 // orders; first plane of the primary top layer
  int npx, nsx;                    // element columns per x row (primary, secondary)
  int ncf;                         // listed coarse faces
  int max_ff;                      // most fine faces on one coarse face
  const int* cf_col;               // [ncf] coarse face column mx + nsx*my
  const int* cf_ptr;               // [ncf+1] fine faces of each coarse face
  const int* ff_col;               // fine face column ex + npx*ey
  const int* ff_sx;                // sub-face interpolation table index (x)
  const int* ff_sy;                // (y)
  int q;                           // Gauss points per direction
  const T* Lp;                     // [q][Np+1] fine GLL basis at the Gauss points
  const T* Ls;                     // [nsub][q][Ns+1] coarse GLL basis at mapped points
  const T* Wq;                     // [q*q] w_qx w_qy |J_F+|
  const T* dp;                     // [Np+1] (2/hz+) l_c'(+1)
  const T* ds;                     // [Ns+1] (2/hz-) l_c'(-1)
  T cp2, cm2, gamma;
  T* Rap; T* Rbp;                  // [B][npx*npy][(Np+1)^2]
  T* Ras; T* Rbs;                  // [B][nsx*nsy][(Ns+1)^2]
  long long rbp, rbs;              // batch strides of the residual arrays
};

// ---------------------------------------------------------------------------
// Face assembly, once per step before the volume launches: the per-face
// interface residuals summed at each face node in a fixed order, and the
// PMUT forcing summed at each node of Gamma_PMUT's face lattice.
// ---------------------------------------------------------------------------
template <typename T>
struct FaceAsmArgs {
  const T* Ra; const T* Rb;        // [B][ne0*ne1][(N+1)^2] per face column
  T* ga; T* gb;                    // [B][L1][py] per face node
  int N, ne0, ne1, L0, L1, py;
  long long rbs, gbs;
};
struct PmutForceArgs {
  const int* node_ptr;             // [L0*L1 + 1] footprint entries of each face node
  const int* node_ent;             // entry ids
  const int* ent_pmut;             // PMUT of each entry
  const double* Bm;                // [nnz][M]: W_face * U.n
  const double* qdd;               // [B][K][M]: q'' of this step
  const float* Bm32;               // FP32 copies (the FP32 state sums f in FP32)
  const float* qdd32;
  int K, M, L0, L1, py;
  double kappa;
  void* f;                         // [B][L1][py] -kappa sum q'' B, state precision
  long long fbs;
};

#ifdef __CUDACC__
// Sum of the per-face (unassembled) interface residual entries touching face
// node (i, j), in a fixed order (deterministic, no atomics).
template <typename T, int N>
__device__ __forceinline__ T face_gather(const T* __restrict__ R, int i, int j, int ne0, int ne1) {
  int fx = i / N, ax = i - fx * N;
  int fy = j / N, ay = j - fy * N;
  if (fx == ne0) { fx = ne0 - 1; ax = N; }
  if (fy == ne1) { fy = ne1 - 1; ay = N; }
  constexpr int F = (N + 1) * (N + 1);
  T s = R[(long long)(fy * ne0 + fx) * F + ay * (N + 1) + ax];
  if (ax == 0 && fx > 0) s += R[(long long)(fy * ne0 + fx - 1) * F + ay * (N + 1) + N];
  if (ay == 0 && fy > 0) s += R[(long long)((fy - 1) * ne0 + fx) * F + N * (N + 1) + ax];
  if (ax == 0 && fx > 0 && ay == 0 && fy > 0) s += R[(long long)((fy - 1) * ne0 + fx - 1) * F + N * (N + 1) + N];
  return s;
}
#endif

// ---------------------------------------------------------------------------
// Perfectly matched layer, one CTA per (layer element, batch member): Phi
// update at the element's GLL nodes and the element residual G Phi^{n+1}.
// ---------------------------------------------------------------------------
template <typename T>
struct PmlArgs {
  const T* p;                      // p^{n+1}, lattice layout
  const T* psi;                    // psi^{n+1/2}, lattice layout
  T* phi;                          // [B][npml][3][(N+1)^3] Phi at half steps, updated in place
  T* r;                            // [B][npml][(N+1)^3] G (Phi^{n+1/2} + Phi^{n+3/2}) / 2
  const int* elem;                 // [npml] element ex + ne0 * (ey + ne1 * ez)
  int npml, N, ne0, ne1;
  int py; long long pz, bstride;
  long long phi_bs, r_bs;
  const T* zeta[3];
  T D[DG_MAXN + 1][DG_MAXN + 1];   // D[i][j] = l_j'(xi_i) of the GLL basis
  T w[DG_MAXN + 1];                // GLL weights
  T g[3];                          // 2 / h_d
  T detJ, c2, dt;
};

// ---------------------------------------------------------------------------
// PMUT modal step (Algorithm 1, PMUT rows) + receiver sampling.
// ---------------------------------------------------------------------------
template <typename T>
struct PmutArgs {
  int B, K, M;
  const int* fp_ptr;               // [K+1] footprint entries of PMUT k
  const long long* fp_off;         // [nnz] offset of the face node in the primary array
  const double* Bm;                // [nnz][M]
  const float* Bm32;               // FP32 copy of Bm: FP32 state, projection sums in FP32; or NULL
  const T* p_prev;                 // p^n of the primary box
  long long bsp;
  double* q; double* qd; double* qdd;   // [B][K][M]
  float* qdd32;                    // FP32 copy of q'' for the forcing assembly, or NULL
  const double* omega2;            // [K][M]
  const double* twozw;             // [K][M] 2 zeta omega
  const double* inv_mu;            // [K][M]
  const double* eta;               // [K][M]
  const double* drive;             // drive[b*dbs + k*dks + n]
  long long dbs, dks;
  int n;                           // step offset inside this run
  const int* step;                 // device step counter of the run (added to n)
  // TX -> RX switch (eq. ode row 2): from absolute step rx_switch on, the
  // voltage is rx_gain[k] sum_m eta_km q_km^n (rx_gain = s / C_k) instead of the drive
  const double* rx_gain;           // [K], or NULL: transmit only
  long long rx_switch;
  const long long* step_base;      // steps done before this run (since rest)
  double* volt;                    // volt[b*vbs + k*vks + n]: voltage used in step n, or NULL
  long long vbs, vks;
  double dt;
  // receivers
  int R;
  int rstride;                     // weights per receiver slot
  const double* rw;                // [R][rstride]
  const long long* roff;           // [R][rstride]
  const int* rdom;                 // [R]
  const int* rnn;                  // [R]
  const T* pc0; const T* pc1;      // p^{n+1} of each box
  long long bs0, bs1;
  double* traces;                  // traces[b*tbs + r*trs + n]
  long long tbs, trs;
};

// Runtime description of one volume launch (FP64 tables, runtime order N);
// the kernel translation unit converts it to VolArgs<T, N>.
struct VolSpec {
  const CUtensorMap* tmap;         // tensor map of p_in
  const CUtensorMap* tmap_v;       // tensor map of v (NULL when the variant does not stage v)
  const CUtensorMap* tmap_pst;     // tensor map of p_out with the v box (TMA-store variants), else NULL
  int* err;
  int* step;                       // step counter to advance (last launch of a step), or NULL
  const void* p_in; void* p_out; void* v;
  long long bstride;
  int L[3], ne[3];
  int py; long long pz;
  double dtv, dtp;
  int N;
  double c[3][DG_MAXN + 1][DG_MAXN + 1];
  double l[3][DG_MAXN + 1], r[3][DG_MAXN + 1];
  double iwv, iwb, iwa[DG_MAXN + 1];
  double minv_scale;
  int has_pmut;
  const void* fpm;
  int iface_k0, iface_top;
  const void* ga; const void* gb;
  long long gbs;
  double dI[DG_MAXN + 1];
  // first-order absorbing sides (x-, x+, y-, y+, z-, z+): C_ii / M_ii of a
  // node on that side, c (2/h_d) / w_0; 0 = rigid wall
  double abc[6];
  int has_abc;
  // perfectly matched layer (see VolArgs); pointers in the state precision
  int has_pml, pml_init;
  const void* zeta[3];
  void* psi;
  const void* rpml;
  const int* pml_slot;
  long long rpml_bs;
  int pml_lo[3], pml_hi[3];
  int layers_per_cta;              // 0: choose automatically
  int tile;                        // tile-shape variant (see vol_impl.cuh)
  int* shape_out;                  // if not NULL: [8] grid xyz, block xyz, layers per CTA, z chunks of the launch
};

// Box shapes (x, y, z) of the TMA staging loads of one element layer (p)
// and of its v planes (vbox, all zero when v is not staged) for a box of
// order N and tile variant `tile`; returns the number of tile variants of
// that order (0 if the order or the variant is unsupported).
int vol_tma_box_f32(int N, int tile, unsigned box[3], unsigned vbox[3]);
int vol_tma_box_f64(int N, int tile, unsigned box[3], unsigned vbox[3]);

// Launchers (defined in the kernel translation units)
// (one instantiation per precision and open-boundary flag, each in its own
// translation unit; the flag removes the absorbing-side and PML terms from
// boxes without them)
template <typename T, bool ABC>
cudaError_t launch_vol_flag(const VolSpec& spec, int batch, cudaStream_t s);
template <typename T>
inline cudaError_t launch_vol(const VolSpec& spec, int batch, cudaStream_t s) {
  return (spec.has_abc || spec.has_pml) ? launch_vol_flag<T, true>(spec, batch, s)
                                         : launch_vol_flag<T, false>(spec, batch, s);
}
template <typename T>
cudaError_t launch_iface(const IfaceArgs<T>& a, int batch, cudaStream_t s);
template <typename T>
cudaError_t launch_pmut_recv(const PmutArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_pml(const PmlArgs<T>& a, int batch, cudaStream_t s);
// one warp waiting on an mbarrier nothing arrives at (bounded; sets *err = 3)
// Sets *flag to 1 if any of x[0..n) is not finite (NaN or Inf); *flag is
// left unchanged otherwise.
cudaError_t launch_nonfinite(const double* x, size_t n, int* flag, cudaStream_t s);
cudaError_t launch_wait_probe(int* err, long long budget, cudaStream_t s);
template <typename T>
cudaError_t launch_face_asm(const FaceAsmArgs<T>& a, int batch, cudaStream_t s);
template <typename T>
cudaError_t launch_pmut_force(const PmutForceArgs& a, int batch, cudaStream_t s);
// power-iteration helpers (FP64)
cudaError_t launch_mdot(const double* x, const double* y, const double* wx, const double* wy, const double* wz, int L0,
                        int L1, int L2, int py, long long pz, double scale, double* out, cudaStream_t s);
cudaError_t launch_mdot(const float* x, const double* y, const double* wx, const double* wy, const double* wz, int L0,
                        int L1, int L2, int py, long long pz, double scale, double* out, cudaStream_t s);
cudaError_t launch_scale(double* x, const double* y, double a, long long n, cudaStream_t s);
// y[0..n) = x[0..n) widened to FP64
cudaError_t launch_widen(const float* x, double* y, long long n, cudaStream_t s);
