// Host setup and C ABI of the DG-SEM + reduced-order PMUT explicit step.
//
// Setup (untimed): GLL / Gauss-Legendre tables, the box lattices, the
// stencil rows of the factorised GLL stiffness (eq. Wf_2), the interface
// maps of Sec. 5 (Algorithm 3 face matching), the PMUT membrane matrix of
// eqs. (f_i)/(g_m), receivers and the time step.
// Hot loop: per step, PMUT modal step + receivers (small.cu), interface
// fluxes (small.cu), fused volume update of each box (vol.cu), following
// Algorithm 1 in its two-vector leapfrog form.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dgsem.h"
#include "internal.h"
#include "tables.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? DGSEM_ENOMEM : DGSEM_ECUDA,         \
                  "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

using dgtab::Basis1D;
using dgtab::gauss;
using dgtab::gll;
using dgtab::legendre;

struct Box {
  double o[3], ext[3], h[3], c, rho;
  int ne[3], N, L[3];
  int py;
  long long pz, bstride;
  Basis1D* basis;
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct dgsem_ctx {
  int device = 0;
  int nd = 0;
  Box box[2];
  Basis1D* basis[2] = {nullptr, nullptr};
  double dt = 0.0, dt_stable = 0.0, cfl = 0.0, alpha = 0.0;
  double dt_cfl = 0.0;                     // dt before the absorbing-boundary limit
  bool dt_fixed = false;                   // dt given by the caller (not from cfl)
  long long ndof = 0;
  VolSpec vspec[2];
  int vol_shape[2][8] = {{0}};   // launch shape of each box's volume kernel in the last run
  // interface
  bool has_iface = false;
  int q = 0, nsub = 0;
  int ncf = 0, nff = 0;
  double gamma = 0.0;
  int max_ff = 0;                          // most fine faces on one coarse face
  int* d_cf_col = nullptr; int* d_cf_ptr = nullptr; int* d_ff_col = nullptr;
  int* d_ff_sx = nullptr; int* d_ff_sy = nullptr;
  void* d_tab[2] = {nullptr, nullptr};   // [fp64, fp32] packed Lp | Ls | Wq | dp | ds
  size_t tab_off[5] = {0, 0, 0, 0, 0};
  // PMUT
  std::vector<double> face_xy;
  int K = 0, M = 0, nnz = 0;
  int* d_fp_ptr = nullptr; long long* d_fp_off = nullptr; double* d_Bm = nullptr;
  float* d_Bm32 = nullptr;                 // FP32 copy of d_Bm (FP32 forcing assembly)
  float* d_qdd32 = nullptr;                // FP32 copy of q'' (run state, FP32 runs)
  int* d_node_ptr = nullptr; int* d_node_ent = nullptr; int* d_ent_pmut = nullptr;
  double* d_modal = nullptr;    // omega2 | twozw | inv_mu | eta   [4][K*M]
  double kappa = 0.0;
  // run state
  int prec = -1, batch = 0;
  void* X[2] = {nullptr, nullptr};
  void* Y[2] = {nullptr, nullptr};
  void* V[2] = {nullptr, nullptr};
  void* Ra[2] = {nullptr, nullptr};
  void* Rb[2] = {nullptr, nullptr};
  double* q_state = nullptr;    // q | qd | qdd  [3][B*K*M]
  long long step = 0;
  // perfectly matched layer per box
  bool has_pml[2] = {false, false};
  std::vector<double> zeta_h[2][3];        // host profiles zeta_d[L_d]
  void* d_zeta[2][2][3] = {};              // [box][fp64, fp32][axis]
  int* d_pml_slot[2] = {nullptr, nullptr}; // [ne2][ne1][ne0] slot or -1
  int* d_pml_elem[2] = {nullptr, nullptr}; // [npml] element index
  int npml[2] = {0, 0};
  int pml_lo[2][3] = {}, pml_hi[2][3] = {};
  // face arrays assembled each step (run state): interface residual per face
  // node of each box, PMUT forcing per node of the primary's z-min face
  void* Ga[2] = {nullptr, nullptr};
  void* Gb[2] = {nullptr, nullptr};
  void* Fpm = nullptr;
  void* Psi[2] = {nullptr, nullptr};       // psi, lattice layout (run state)
  void* Phi[2] = {nullptr, nullptr};       // [B][npml][3][(N+1)^3] (run state)
  void* Rpml[2] = {nullptr, nullptr};      // [B][npml][(N+1)^3] (run state)
  // TX -> RX switch of the PMUT array (off: rx_switch < 0)
  long long rx_switch = -1;
  double* d_rx_gain = nullptr;             // [K] s / C_k
  long long* d_step_base = nullptr;        // steps done before the current run
  double* d_volt = nullptr;                // [B][K][S] voltages of the last run
  size_t volt_cap = 0;
  long long volt_n = 0;                    // doubles recorded by the last run
  bool state_valid = false;
  // pending initial state
  std::vector<double> init_p, init_v;
  bool has_init = false;
  // scratch for host-pointer runs
  double* d_drive = nullptr; size_t drive_cap = 0;
  double* d_traces = nullptr; size_t traces_cap = 0;
  double* d_rw = nullptr; long long* d_roff = nullptr; int* d_rdom = nullptr; int* d_rnn = nullptr;
  size_t recv_cap = 0;
  // TMA descriptors of the pressure buffers (X and Y of each box) and the
  // device status word written by bounded waits
  CUtensorMap tmap_x[2], tmap_y[2], tmap_v[2];
  CUtensorMap tmap_px[2], tmap_py[2];   // X / Y with the v box: p_out of the TMA-store tile variants
  bool has_tmap_v[2] = {false, false};
  int tile_pref[2][2] = {{0, 0}, {0, 0}};   // [fp64, fp32][box] tile-shape variant
  int* d_err = nullptr;
  int* d_nf = nullptr;                        // non-finite flag of the divergence check
  int* d_step = nullptr;                      // step counter of the current run
  // CUDA graph of a block of steps, replayed by dgsem_run
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream = nullptr;      // second branch of a captured step
  cudaEvent_t fork_ev[2] = {nullptr, nullptr};
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  long long graph_launches[DGSEM_K_COUNT] = {};
  std::vector<unsigned char> graph_key;
  // instrumentation
  bool profiling = false;
  long long launches[DGSEM_K_COUNT] = {};
  double kernel_ms[DGSEM_K_COUNT] = {};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;   // (kind, index of start event; stop = index + 1)
};

namespace {

template <typename P>
int dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return DGSEM_OK;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(DGSEM_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  return DGSEM_OK;
}

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

template <typename V>
int upload(V** d, const std::vector<V>& h) {
  int rc = dalloc(d, h.size() * sizeof(V));
  if (rc) return rc;
  if (!h.empty()) CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
  return DGSEM_OK;
}

void drop_graph(dgsem_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_key.clear();
}

void free_run_state(dgsem_ctx* c) {
  drop_graph(c);
  for (int d = 0; d < 2; ++d) {
    dfree(c->X[d]); dfree(c->Y[d]); dfree(c->V[d]); dfree(c->Ra[d]); dfree(c->Rb[d]);
    dfree(c->Psi[d]); dfree(c->Phi[d]); dfree(c->Rpml[d]);
    dfree(c->Ga[d]); dfree(c->Gb[d]);
  }
  dfree(c->Fpm);
  dfree(c->d_qdd32);
  dfree(c->q_state);
  c->prec = -1;
  c->batch = 0;
  c->state_valid = false;
}

size_t elem_size(int prec) { return prec == DGSEM_FP32_MIXED ? sizeof(float) : sizeof(double); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 4D (x, y, z, batch) tiled tensor map of one state buffer of a box for the
// TMA staging loads of the volume kernel (box = one element layer of a tile).
int make_tmap(CUtensorMap* out, void* base, const Box& B, int batch, int prec, const unsigned box[3]) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(DGSEM_ECUDA, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const size_t es = elem_size(prec);
  if (!box[0] || !box[1] || !box[2]) return fail(DGSEM_EINVAL, "empty TMA box");
  if ((box[0] * es) % 16) return fail(DGSEM_EINVAL, "TMA box row not a multiple of 16 bytes");
  const cuuint64_t dims[4] = {(cuuint64_t)B.L[0], (cuuint64_t)B.L[1], (cuuint64_t)B.L[2], (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)B.py * es, (cuuint64_t)B.pz * es, (cuuint64_t)B.bstride * es};
  for (int i = 0; i < 3; ++i)
    if (strides[i] % 16) return fail(DGSEM_EINVAL, "TMA stride %d not a multiple of 16 bytes", i);
  if (reinterpret_cast<uintptr_t>(base) % 16) return fail(DGSEM_EINVAL, "TMA base address not 16-byte aligned");
  const cuuint32_t boxd[4] = {box[0], box[1], box[2], 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(out, prec == DGSEM_FP32_MIXED ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                      4, base, dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(DGSEM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGSEM_OK;
}

int ensure_run_state(dgsem_ctx* c, int prec, int batch) {
  if (c->prec == prec && c->batch == batch && c->X[0]) return DGSEM_OK;
  free_run_state(c);
  const size_t es = elem_size(prec);
  for (int d = 0; d < c->nd; ++d) {
    const size_t bytes = (size_t)batch * c->box[d].bstride * es;
    int rc;
    if ((rc = dalloc(&c->X[d], bytes)) || (rc = dalloc(&c->Y[d], bytes)) || (rc = dalloc(&c->V[d], bytes))) {
      free_run_state(c);
      return rc;
    }
    if (c->has_iface) {
      const Box& B = c->box[d];
      const size_t rb = (size_t)batch * B.ne[0] * B.ne[1] * (B.N + 1) * (B.N + 1) * es;
      if ((rc = dalloc(&c->Ra[d], rb)) || (rc = dalloc(&c->Rb[d], rb))) {
        free_run_state(c);
        return rc;
      }
      CUDA_TRY(cudaMemset(c->Ra[d], 0, rb));
      CUDA_TRY(cudaMemset(c->Rb[d], 0, rb));
      const size_t gb = (size_t)batch * B.L[1] * B.py * es;
      if ((rc = dalloc(&c->Ga[d], gb)) || (rc = dalloc(&c->Gb[d], gb))) {
        free_run_state(c);
        return rc;
      }
      CUDA_TRY(cudaMemset(c->Ga[d], 0, gb));
      CUDA_TRY(cudaMemset(c->Gb[d], 0, gb));
    }
    if (c->has_pml[d]) {
      const Box& B = c->box[d];
      const size_t nl = (size_t)(B.N + 1) * (B.N + 1) * (B.N + 1);
      const size_t fb = (size_t)batch * c->npml[d] * 3 * nl * es, rb = (size_t)batch * c->npml[d] * nl * es;
      if ((rc = dalloc(&c->Psi[d], bytes)) || (rc = dalloc(&c->Phi[d], fb)) || (rc = dalloc(&c->Rpml[d], rb))) {
        free_run_state(c);
        return rc;
      }
    }
  }
  if (c->K > 0) {
    int rc = dalloc(&c->q_state, (size_t)3 * batch * c->K * c->M * sizeof(double));
    if (!rc && prec == DGSEM_FP32_MIXED) rc = dalloc(&c->d_qdd32, (size_t)batch * c->K * c->M * sizeof(float));
    const size_t fb = (size_t)batch * c->box[0].L[1] * c->box[0].py * es;
    if (!rc) rc = dalloc(&c->Fpm, fb);
    if (rc) { free_run_state(c); return rc; }
    CUDA_TRY(cudaMemset(c->Fpm, 0, fb));
  }
  c->prec = prec;
  c->batch = batch;
  c->state_valid = false;
  return DGSEM_OK;
}

// (Re-)encode the TMA descriptors of both pressure buffers of every box for
// the tile variants selected for the current precision.
int refresh_tmaps(dgsem_ctx* c) {
  for (int d = 0; d < c->nd; ++d) {
    const int tile = c->tile_pref[c->prec == DGSEM_FP32_MIXED ? 1 : 0][d];
    unsigned box[3], vbox[3];
    const int nv = c->prec == DGSEM_FP32_MIXED ? vol_tma_box_f32(c->box[d].N, tile, box, vbox)
                                               : vol_tma_box_f64(c->box[d].N, tile, box, vbox);
    if (!nv) return fail(DGSEM_EINVAL, "no tile variant %d for order %d", tile, c->box[d].N);
    int rc;
    if ((rc = make_tmap(&c->tmap_x[d], c->X[d], c->box[d], c->batch, c->prec, box)) ||
        (rc = make_tmap(&c->tmap_y[d], c->Y[d], c->box[d], c->batch, c->prec, box)))
      return rc;
    c->has_tmap_v[d] = vbox[0] != 0;
    if (c->has_tmap_v[d] && ((rc = make_tmap(&c->tmap_v[d], c->V[d], c->box[d], c->batch, c->prec, vbox)) ||
                             (rc = make_tmap(&c->tmap_px[d], c->X[d], c->box[d], c->batch, c->prec, vbox)) ||
                             (rc = make_tmap(&c->tmap_py[d], c->Y[d], c->box[d], c->batch, c->prec, vbox))))
      return rc;
  }
  return DGSEM_OK;
}

int zero_state(dgsem_ctx* c, cudaStream_t s) {
  const size_t es = elem_size(c->prec);
  for (int d = 0; d < c->nd; ++d) {
    const size_t bytes = (size_t)c->batch * c->box[d].bstride * es;
    CUDA_TRY(cudaMemsetAsync(c->X[d], 0, bytes, s));
    CUDA_TRY(cudaMemsetAsync(c->Y[d], 0, bytes, s));
    CUDA_TRY(cudaMemsetAsync(c->V[d], 0, bytes, s));
  }
  if (c->q_state)
    CUDA_TRY(cudaMemsetAsync(c->q_state, 0, (size_t)3 * c->batch * c->K * c->M * sizeof(double), s));
  for (int d = 0; d < c->nd; ++d) {
    if (!c->has_pml[d]) continue;
    const Box& B = c->box[d];
    const size_t nl = (size_t)(B.N + 1) * (B.N + 1) * (B.N + 1);
    CUDA_TRY(cudaMemsetAsync(c->Psi[d], 0, (size_t)c->batch * B.bstride * es, s));
    CUDA_TRY(cudaMemsetAsync(c->Phi[d], 0, (size_t)c->batch * c->npml[d] * 3 * nl * es, s));
  }
  c->step = 0;
  return DGSEM_OK;
}

// Build the stencil rows of one box (see VolArgs).
void build_vol_spec(const Box& B, VolSpec& v) {
  std::memset(&v, 0, sizeof(v));
  const Basis1D& bs = *B.basis;
  const int N = B.N;
  v.N = N;
  for (int d = 0; d < 3; ++d) {
    v.L[d] = B.L[d];
    v.ne[d] = B.ne[d];
    const double s = B.c * B.c * (2.0 / B.h[d]) * (2.0 / B.h[d]);
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N; ++b) v.c[d][a][b] = (a > 0 && a < N) ? s * bs.A[a * (N + 1) + b] / bs.w[a] : 0.0;
    for (int b = 0; b <= N; ++b) {
      v.l[d][b] = s * bs.A[N * (N + 1) + b];
      v.r[d][b] = s * bs.A[0 * (N + 1) + b];
    }
  }
  v.iwv = 1.0 / (bs.w[0] + bs.w[N]);
  v.iwb = 1.0 / bs.w[0];
  for (int a = 0; a <= N; ++a) v.iwa[a] = 1.0 / bs.w[a];
  v.minv_scale = 8.0 / (B.h[0] * B.h[1] * B.h[2]);
  v.py = B.py;
  v.pz = B.pz;
  v.bstride = B.bstride;
  v.iface_k0 = -1;
}

// ---------------------------------------------------------------------------
// Interface setup: Algorithm 3 (normal filter, one-vertex radius filter,
// inverse map), on a bucket grid of the coarse faces' stored vertices.
// ---------------------------------------------------------------------------
int build_interface(dgsem_ctx* c, const dgsem_mesh_desc* desc) {
  const Box& P = c->box[0];
  const Box& S = c->box[1];
  const double tol = 1e-9 * std::max(P.ext[0], P.ext[1]);
  if (std::fabs(S.o[2] - (P.o[2] + P.ext[2])) > tol || std::fabs(S.o[0] - P.o[0]) > tol ||
      std::fabs(S.o[1] - P.o[1]) > tol || std::fabs(S.ext[0] - P.ext[0]) > tol ||
      std::fabs(S.ext[1] - P.ext[1]) > tol)
    return fail(DGSEM_EINVAL, "secondary box must sit on the primary's z-max face with the same x-y extent");
  std::vector<int> fine, coarse;
  if (desc->fine_faces) {
    if (desc->n_fine_faces < 0) return fail(DGSEM_EINVAL, "n_fine_faces < 0");
    fine.assign(desc->fine_faces, desc->fine_faces + desc->n_fine_faces);
  } else {
    for (int i = 0; i < P.ne[0] * P.ne[1]; ++i) fine.push_back(i);
  }
  if (desc->coarse_faces) {
    if (desc->n_coarse_faces < 0) return fail(DGSEM_EINVAL, "n_coarse_faces < 0");
    coarse.assign(desc->coarse_faces, desc->coarse_faces + desc->n_coarse_faces);
  } else {
    for (int i = 0; i < S.ne[0] * S.ne[1]; ++i) coarse.push_back(i);
  }
  for (int f : fine)
    if (f < 0 || f >= P.ne[0] * P.ne[1]) return fail(DGSEM_EINVAL, "fine face %d out of range", f);
  for (int f : coarse)
    if (f < 0 || f >= S.ne[0] * S.ne[1]) return fail(DGSEM_EINVAL, "coarse face %d out of range", f);
  const int q = desc->iface_quad_pts > 0 ? desc->iface_quad_pts : std::max(P.N, S.N) + 1;
  if (q > DG_MAXQ) return fail(DGSEM_EINVAL, "iface_quad_pts %d > %d", q, DG_MAXQ);
  c->q = q;
  std::vector<double> gx, gw;
  gauss(q, gx, gw);
  // coarse faces: stored vertex (x-min, y-min corner), normal -e_z, diameter
  const double hs0 = S.h[0], hs1 = S.h[1];
  const double diam_c = std::sqrt(hs0 * hs0 + hs1 * hs1);
  const double diam_f = std::sqrt(P.h[0] * P.h[0] + P.h[1] * P.h[1]);
  const double radius = std::max(diam_c, diam_f) * (1.0 + 1e-9);
  std::map<long long, std::vector<int>> bucket;   // bucket of the stored vertex -> coarse list index
  for (size_t i = 0; i < coarse.size(); ++i) {
    const int mx = coarse[i] % S.ne[0], my = coarse[i] / S.ne[0];
    bucket[(long long)my * (S.ne[0] + 1) + mx].push_back((int)i);
  }
  const double n_plus[3] = {0.0, 0.0, 1.0}, n_minus[3] = {0.0, 0.0, -1.0};
  std::vector<std::vector<int>> by_coarse(coarse.size());
  std::vector<double> off_x(fine.size()), off_y(fine.size());
  std::vector<int> match(fine.size(), -1);
  for (size_t f = 0; f < fine.size(); ++f) {
    const int ex = fine[f] % P.ne[0], ey = fine[f] / P.ne[0];
    const double fx0 = P.o[0] + ex * P.h[0], fy0 = P.o[1] + ey * P.h[1];
    int found = -1;
    for (int qy = 0; qy < q; ++qy)
      for (int qx = 0; qx < q; ++qx) {
        const double x = fx0 + 0.5 * (gx[qx] + 1.0) * P.h[0];
        const double y = fy0 + 0.5 * (gx[qy] + 1.0) * P.h[1];
        const int bx = (int)std::floor((x - S.o[0]) / hs0), by = (int)std::floor((y - S.o[1]) / hs1);
        int hit = -1;
        for (int dy = -2; dy <= 2 && hit < 0; ++dy)
          for (int dx = -2; dx <= 2 && hit < 0; ++dx) {
            auto it = bucket.find((long long)(by + dy) * (S.ne[0] + 1) + (bx + dx));
            if (it == bucket.end()) continue;
            for (int ci : it->second) {
              double nn = 0.0;
              for (int d = 0; d < 3; ++d) nn += (n_plus[d] + n_minus[d]) * (n_plus[d] + n_minus[d]);
              if (std::sqrt(nn) >= 1e-9) continue;                      // normal filter
              const int mx = coarse[ci] % S.ne[0], my = coarse[ci] / S.ne[0];
              const double vx = S.o[0] + mx * hs0, vy = S.o[1] + my * hs1;
              if (std::hypot(vx - x, vy - y) > radius) continue;        // radius filter
              // inverse map of the affine coarse element: reference coordinates
              const double rx = 2.0 * (x - vx) / hs0 - 1.0, ry = 2.0 * (y - vy) / hs1 - 1.0;
              if (std::fabs(rx) <= 1.0 + 1e-10 && std::fabs(ry) <= 1.0 + 1e-10) { hit = ci; break; }
            }
          }
        if (hit < 0) return fail(DGSEM_ENOMATCH, "fine face %d: quadrature node without a coarse neighbour", fine[f]);
        if (found >= 0 && hit != found)
          return fail(DGSEM_ENOMATCH, "fine face %d straddles two coarse faces", fine[f]);
        found = hit;
      }
    match[f] = found;
    by_coarse[found].push_back((int)f);
    const int mx = coarse[found] % S.ne[0], my = coarse[found] / S.ne[0];
    // affine sub-face map x^- = s x^+ + o along each axis
    off_x[f] = (2.0 * (fx0 - (S.o[0] + mx * hs0)) + P.h[0]) / hs0 - 1.0;
    off_y[f] = (2.0 * (fy0 - (S.o[1] + my * hs1)) + P.h[1]) / hs1 - 1.0;
  }
  const double sx = P.h[0] / hs0, sy = P.h[1] / hs1;
  // distinct affine sub-face maps (scale, offset) -> interpolation tables Ls[nsub][q][Ns+1]
  std::vector<double> offs, scales;
  auto sub_index = [&](double o, double sc) {
    for (size_t i = 0; i < offs.size(); ++i)
      if (std::fabs(offs[i] - o) < 1e-12 && std::fabs(scales[i] - sc) < 1e-12) return (int)i;
    offs.push_back(o);
    scales.push_back(sc);
    return (int)offs.size() - 1;
  };
  std::vector<int> h_cf_col, h_cf_ptr(1, 0), h_ff_col, h_ff_sx, h_ff_sy;
  for (size_t ci = 0; ci < coarse.size(); ++ci) {
    if (by_coarse[ci].empty()) continue;
    h_cf_col.push_back(coarse[ci]);
    for (int f : by_coarse[ci]) {
      h_ff_col.push_back(fine[f]);
      h_ff_sx.push_back(sub_index(off_x[f], sx));
      h_ff_sy.push_back(sub_index(off_y[f], sy));
    }
    h_cf_ptr.push_back((int)h_ff_col.size());
  }
  c->ncf = (int)h_cf_col.size();
  c->nff = (int)h_ff_col.size();
  c->max_ff = 0;
  for (size_t i = 0; i + 1 < h_cf_ptr.size(); ++i) c->max_ff = std::max(c->max_ff, h_cf_ptr[i + 1] - h_cf_ptr[i]);
  c->nsub = (int)offs.size();
  const int np1 = P.N + 1, ns1 = S.N + 1;
  std::vector<double> Lp(q * np1), Ls(offs.size() * q * ns1), Wq(q * q), dp(np1), ds(ns1);
  for (int t = 0; t < q; ++t) P.basis->values(gx[t], &Lp[t * np1]);
  for (size_t si = 0; si < offs.size(); ++si)
    for (int t = 0; t < q; ++t) S.basis->values(scales[si] * gx[t] + offs[si], &Ls[(si * q + t) * ns1]);
  const double jac = P.h[0] * P.h[1] / 4.0;
  for (int ty = 0; ty < q; ++ty)
    for (int tx = 0; tx < q; ++tx) Wq[ty * q + tx] = gw[tx] * gw[ty] * jac;
  for (int cc = 0; cc < np1; ++cc) dp[cc] = (2.0 / P.h[2]) * P.basis->D[P.N * np1 + cc];
  for (int cc = 0; cc < ns1; ++cc) ds[cc] = (2.0 / S.h[2]) * S.basis->D[0 * ns1 + cc];
  const double cbar = 2.0 * P.c * S.c / (P.c + S.c);
  c->gamma = c->alpha * cbar * cbar * std::max(P.N, S.N) * std::max(P.N, S.N) / std::min(P.h[2], S.h[2]);
  // packed tables, FP64 and FP32 copies
  std::vector<double> tab;
  c->tab_off[0] = 0; tab.insert(tab.end(), Lp.begin(), Lp.end());
  c->tab_off[1] = tab.size(); tab.insert(tab.end(), Ls.begin(), Ls.end());
  c->tab_off[2] = tab.size(); tab.insert(tab.end(), Wq.begin(), Wq.end());
  c->tab_off[3] = tab.size(); tab.insert(tab.end(), dp.begin(), dp.end());
  c->tab_off[4] = tab.size(); tab.insert(tab.end(), ds.begin(), ds.end());
  std::vector<float> tabf(tab.begin(), tab.end());
  int rc;
  if ((rc = upload((double**)&c->d_tab[0], tab)) || (rc = upload((float**)&c->d_tab[1], tabf)) ||
      (rc = upload(&c->d_cf_col, h_cf_col)) || (rc = upload(&c->d_cf_ptr, h_cf_ptr)) ||
      (rc = upload(&c->d_ff_col, h_ff_col)) || (rc = upload(&c->d_ff_sx, h_ff_sx)) ||
      (rc = upload(&c->d_ff_sy, h_ff_sy)))
    return rc;
  // residual layout for the volume kernels
  c->vspec[0].iface_k0 = (P.ne[2] - 1) * P.N;
  c->vspec[0].iface_top = 1;
  for (int cc = 0; cc < np1; ++cc) c->vspec[0].dI[cc] = dp[cc];
  c->vspec[1].iface_k0 = 0;
  c->vspec[1].iface_top = 0;
  for (int cc = 0; cc < ns1; ++cc) c->vspec[1].dI[cc] = ds[cc];
  c->has_iface = true;
  return DGSEM_OK;
}

template <typename T>
IfaceArgs<T> iface_args(const dgsem_ctx* c) {
  IfaceArgs<T> a;
  const Box& P = c->box[0];
  const Box& S = c->box[1];
  const int pi = sizeof(T) == 8 ? 0 : 1;
  const T* tab = static_cast<const T*>(c->d_tab[pi]);
  a.pp = static_cast<const T*>(c->Y[0]);
  a.ps = static_cast<const T*>(c->Y[1]);
  a.bsp = P.bstride; a.bss = S.bstride;
  a.pyp = P.py; a.pzp = P.pz; a.pys = S.py; a.pzs = S.pz;
  a.Np = P.N; a.Ns = S.N; a.kp0 = (P.ne[2] - 1) * P.N;
  a.npx = P.ne[0]; a.nsx = S.ne[0];
  a.ncf = c->ncf;
  a.max_ff = c->max_ff;
  a.cf_col = c->d_cf_col; a.cf_ptr = c->d_cf_ptr; a.ff_col = c->d_ff_col;
  a.ff_sx = c->d_ff_sx; a.ff_sy = c->d_ff_sy;
  a.q = c->q;
  a.Lp = tab + c->tab_off[0]; a.Ls = tab + c->tab_off[1]; a.Wq = tab + c->tab_off[2];
  a.dp = tab + c->tab_off[3]; a.ds = tab + c->tab_off[4];
  a.cp2 = T(P.c * P.c); a.cm2 = T(S.c * S.c); a.gamma = T(c->gamma);
  a.Rap = static_cast<T*>(c->Ra[0]); a.Rbp = static_cast<T*>(c->Rb[0]);
  a.Ras = static_cast<T*>(c->Ra[1]); a.Rbs = static_cast<T*>(c->Rb[1]);
  a.rbp = (long long)P.ne[0] * P.ne[1] * (P.N + 1) * (P.N + 1);
  a.rbs = (long long)S.ne[0] * S.ne[1] * (S.N + 1) * (S.N + 1);
  return a;
}

// Bracket a kernel launch with events when profiling (events from a pool).
struct LaunchTimer {
  dgsem_ctx* c; cudaStream_t s; int kind; int idx = -1;
  LaunchTimer(dgsem_ctx* c_, cudaStream_t s_, int kind_) : c(c_), s(s_), kind(kind_) {
    c->launches[kind]++;
    if (!c->profiling) return;
    idx = 2 * (int)c->ev_used.size();
    while ((int)c->ev_pool.size() < idx + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { idx = -1; return; }
      c->ev_pool.push_back(e);
    }
    cudaEventRecord(c->ev_pool[idx], s);
  }
  ~LaunchTimer() {
    if (idx < 0) return;
    cudaEventRecord(c->ev_pool[idx + 1], s);
    c->ev_used.push_back({kind, idx});
  }
};

void collect_timings(dgsem_ctx* c) {
  for (auto& u : c->ev_used) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[u.second], c->ev_pool[u.second + 1]) == cudaSuccess)
      c->kernel_ms[u.first] += ms;
  }
  c->ev_used.clear();
}

// Assemble the face arrays the volume launches read: the interface residual
// of every face node of each box (after the interface launch) and, when
// pmut, the PMUT forcing of the primary's z-min face (after the PMUT launch).
template <typename T>
int launch_face_assembly(dgsem_ctx* c, cudaStream_t s, int batch, bool pmut) {
  if (c->has_iface) {
    for (int d = 0; d < c->nd; ++d) {
      const Box& B = c->box[d];
      FaceAsmArgs<T> a;
      a.Ra = static_cast<const T*>(c->Ra[d]); a.Rb = static_cast<const T*>(c->Rb[d]);
      a.ga = static_cast<T*>(c->Ga[d]); a.gb = static_cast<T*>(c->Gb[d]);
      a.N = B.N; a.ne0 = B.ne[0]; a.ne1 = B.ne[1]; a.L0 = B.L[0]; a.L1 = B.L[1]; a.py = B.py;
      a.rbs = (long long)B.ne[0] * B.ne[1] * (B.N + 1) * (B.N + 1);
      a.gbs = (long long)B.L[1] * B.py;
      LaunchTimer lt(c, s, DGSEM_K_IFACE);
      CUDA_TRY(launch_face_asm<T>(a, batch, s));
    }
  }
  if (pmut && c->K > 0) {
    const Box& P = c->box[0];
    PmutForceArgs a;
    a.node_ptr = c->d_node_ptr; a.node_ent = c->d_node_ent; a.ent_pmut = c->d_ent_pmut;
    a.Bm = c->d_Bm; a.qdd = c->q_state + 2LL * batch * c->K * c->M;
    a.Bm32 = c->d_Bm32; a.qdd32 = c->d_qdd32;
    a.K = c->K; a.M = c->M; a.L0 = P.L[0]; a.L1 = P.L[1]; a.py = P.py;
    a.kappa = c->kappa;
    a.f = c->Fpm; a.fbs = (long long)P.L[1] * P.py;
    LaunchTimer lt(c, s, DGSEM_K_PMUT_RECV);
    CUDA_TRY(launch_pmut_force<T>(a, batch, s));
  }
  return DGSEM_OK;
}

// One time step (or the initial half step when init is true).  With a side
// stream (graph capture of a two-box mesh) the PMUT/receiver launch runs on
// the side stream, concurrently with the interface launch on s; both volume
// launches follow on s (the primary needs q'' of this step, both need the
// interface residual).  Running the two volume launches concurrently as well
// was measured slower: their CTAs compete for shared memory and bandwidth.
// Without a side stream everything runs on s in that order.
template <typename T>
int launch_step(dgsem_ctx* c, cudaStream_t s, const double* drive, long long dbs, long long dks, int n_local,
                int R, double* traces, long long tbs, long long trs, bool init, cudaStream_t side = nullptr,
                double* volt = nullptr) {
  const bool fork = side && c->nd == 2 && c->has_iface && !init;
  cudaStream_t sp = fork ? side : s;       // stream of the PMUT launch
  if (fork) {
    CUDA_TRY(cudaEventRecord(c->fork_ev[0], s));
    CUDA_TRY(cudaStreamWaitEvent(side, c->fork_ev[0], 0));
  }
  if (!init && (c->K > 0 || R > 0)) {
    PmutArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.B = c->batch; a.K = c->K; a.M = c->M;
    a.fp_ptr = c->d_fp_ptr; a.fp_off = c->d_fp_off; a.Bm = c->d_Bm;
    a.qdd32 = std::is_same<T, float>::value ? c->d_qdd32 : nullptr;
    a.Bm32 = std::is_same<T, float>::value ? c->d_Bm32 : nullptr;
    a.p_prev = static_cast<const T*>(c->X[0]);
    a.bsp = c->box[0].bstride;
    const long long kmB = (long long)c->batch * c->K * c->M;
    a.q = c->q_state; a.qd = c->q_state ? c->q_state + kmB : nullptr; a.qdd = c->q_state ? c->q_state + 2 * kmB : nullptr;
    const long long km = (long long)c->K * c->M;
    a.omega2 = c->d_modal; a.twozw = c->d_modal ? c->d_modal + km : nullptr;
    a.inv_mu = c->d_modal ? c->d_modal + 2 * km : nullptr; a.eta = c->d_modal ? c->d_modal + 3 * km : nullptr;
    a.drive = drive; a.dbs = dbs; a.dks = dks; a.n = n_local; a.step = c->d_step; a.dt = c->dt;
    a.R = R; a.rstride = 0;
    if (R > 0) {
      int maxn = 0;
      for (int d = 0; d < c->nd; ++d) maxn = std::max(maxn, (c->box[d].N + 1) * (c->box[d].N + 1) * (c->box[d].N + 1));
      a.rstride = maxn;
    }
    a.rw = c->d_rw; a.roff = c->d_roff; a.rdom = c->d_rdom; a.rnn = c->d_rnn;
    a.pc0 = static_cast<const T*>(c->Y[0]); a.pc1 = c->nd > 1 ? static_cast<const T*>(c->Y[1]) : nullptr;
    a.bs0 = c->box[0].bstride; a.bs1 = c->nd > 1 ? c->box[1].bstride : 0;
    a.traces = traces; a.tbs = tbs; a.trs = trs;
    if (c->rx_switch >= 0) {
      a.rx_gain = c->d_rx_gain; a.rx_switch = c->rx_switch; a.step_base = c->d_step_base;
    }
    a.volt = volt; a.vbs = (long long)c->K * dks; a.vks = dks;
    LaunchTimer lt(c, sp, DGSEM_K_PMUT_RECV);
    CUDA_TRY(launch_pmut_recv<T>(a, sp));
  }
  if (fork) CUDA_TRY(cudaEventRecord(c->fork_ev[1], side));
  // init: p_in = X (p^0), p_out = Y (p^1); step: p_in = Y (p^{n+1}), p_out = X (p^{n+2})
  void* pin[2]; void* pout[2];
  for (int d = 0; d < c->nd; ++d) {
    pin[d] = init ? c->X[d] : c->Y[d];
    pout[d] = init ? c->Y[d] : c->X[d];
  }
  if (c->has_iface) {
    IfaceArgs<T> a = iface_args<T>(c);
    a.pp = static_cast<const T*>(pin[0]);
    a.ps = static_cast<const T*>(pin[1]);
    LaunchTimer lt(c, s, DGSEM_K_IFACE);
    CUDA_TRY(launch_iface<T>(a, c->batch, s));
  }
  if (fork) CUDA_TRY(cudaStreamWaitEvent(s, c->fork_ev[1], 0));
  {
    const int rc = launch_face_assembly<T>(c, s, c->batch, !init);
    if (rc) return rc;
  }
  // perfectly matched layers: Phi update and element residuals (read p^{n+1}, psi^{n+1/2})
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  for (int d = 0; d < c->nd && !init; ++d) {
    if (!c->has_pml[d]) continue;
    const Box& B = c->box[d];
    const int nl = (B.N + 1) * (B.N + 1) * (B.N + 1);
    PmlArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.p = static_cast<const T*>(pin[d]);
    a.psi = static_cast<const T*>(c->Psi[d]);
    a.phi = static_cast<T*>(c->Phi[d]);
    a.r = static_cast<T*>(c->Rpml[d]);
    a.elem = c->d_pml_elem[d];
    a.npml = c->npml[d]; a.N = B.N; a.ne0 = B.ne[0]; a.ne1 = B.ne[1];
    a.py = B.py; a.pz = B.pz; a.bstride = B.bstride;
    a.phi_bs = (long long)c->npml[d] * 3 * nl; a.r_bs = (long long)c->npml[d] * nl;
    for (int ax = 0; ax < 3; ++ax) {
      a.zeta[ax] = static_cast<const T*>(c->d_zeta[d][pi][ax]);
      a.g[ax] = T(2.0 / B.h[ax]);
    }
    for (int i = 0; i <= B.N; ++i) {
      a.w[i] = T(B.basis->w[i]);
      for (int j = 0; j <= B.N; ++j) a.D[i][j] = T(B.basis->D[i * (B.N + 1) + j]);
    }
    a.detJ = T(B.h[0] * B.h[1] * B.h[2] / 8.0);
    a.c2 = T(B.c * B.c);
    a.dt = T(c->dt);
    LaunchTimer lt(c, s, DGSEM_K_PML);
    CUDA_TRY(launch_pml<T>(a, c->batch, s));
  }
  for (int d = 0; d < c->nd; ++d) {
    VolSpec v = c->vspec[d];
    v.tmap = init ? &c->tmap_x[d] : &c->tmap_y[d];
    v.tmap_v = c->has_tmap_v[d] ? &c->tmap_v[d] : nullptr;
    v.tmap_pst = c->has_tmap_v[d] ? (init ? &c->tmap_py[d] : &c->tmap_px[d]) : nullptr;
    v.err = c->d_err;
    v.tile = c->tile_pref[c->prec == DGSEM_FP32_MIXED ? 1 : 0][d];
    v.step = (!init && d == c->nd - 1) ? c->d_step : nullptr;
    v.p_in = pin[d]; v.p_out = pout[d]; v.v = c->V[d];
    v.dtv = init ? 0.5 * c->dt : c->dt;
    v.dtp = c->dt;
    v.ga = c->Ga[d]; v.gb = c->Gb[d];
    v.gbs = (long long)c->box[d].L[1] * c->box[d].py;
    if (c->has_pml[d]) {
      const Box& B = c->box[d];
      v.has_pml = 1;
      v.pml_init = init ? 1 : 0;
      for (int ax = 0; ax < 3; ++ax) {
        v.zeta[ax] = c->d_zeta[d][pi][ax];
        v.pml_lo[ax] = c->pml_lo[d][ax];
        v.pml_hi[ax] = c->pml_hi[d][ax];
      }
      v.psi = c->Psi[d];
      v.rpml = c->Rpml[d];
      v.pml_slot = c->d_pml_slot[d];
      v.rpml_bs = (long long)c->npml[d] * (B.N + 1) * (B.N + 1) * (B.N + 1);
    }
    if (d == 0 && c->K > 0 && !init) {
      v.has_pmut = 1;
      v.fpm = c->Fpm;
    }
    v.shape_out = c->vol_shape[d];
    LaunchTimer lt(c, s, DGSEM_K_VOL0 + d);
    CUDA_TRY(launch_vol<T>(v, c->batch, s));
  }
  if (!init) {
    for (int d = 0; d < c->nd; ++d) {
      std::swap(c->X[d], c->Y[d]);
      std::swap(c->tmap_x[d], c->tmap_y[d]);
      std::swap(c->tmap_px[d], c->tmap_py[d]);
    }
  }
  return DGSEM_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Receivers: containing element (lowest id on ties; primary first), weights.
int setup_receivers(dgsem_ctx* c, int R, const double* xyz) {
  if (R == 0) return DGSEM_OK;
  int maxn = 0;
  for (int d = 0; d < c->nd; ++d) maxn = std::max(maxn, (c->box[d].N + 1) * (c->box[d].N + 1) * (c->box[d].N + 1));
  std::vector<double> w((size_t)R * maxn, 0.0);
  std::vector<long long> off((size_t)R * maxn, 0);
  std::vector<int> dom(R), nn(R);
  for (int r = 0; r < R; ++r) {
    const double* x = xyz + 3 * r;
    int found = -1;
    for (int d = 0; d < c->nd && found < 0; ++d) {
      const Box& B = c->box[d];
      bool inside = true;
      for (int k = 0; k < 3; ++k) {
        const double t = 1e-12 * B.ext[k];
        if (x[k] < B.o[k] - t || x[k] > B.o[k] + B.ext[k] + t) inside = false;
      }
      if (inside) found = d;
    }
    if (found < 0) return fail(DGSEM_EINVAL, "receiver %d at (%g, %g, %g) is outside the mesh", r, x[0], x[1], x[2]);
    const Box& B = c->box[found];
    int e[3];
    double ref[3];
    for (int k = 0; k < 3; ++k) {
      const double u = (x[k] - B.o[k]) / B.h[k];
      int ek = (int)std::ceil(u - 1e-12) - 1;      // lowest element containing the point
      ek = std::max(0, std::min(ek, B.ne[k] - 1));
      e[k] = ek;
      ref[k] = std::max(-1.0, std::min(1.0, 2.0 * (u - ek) - 1.0));
    }
    const int n1 = B.N + 1;
    std::vector<double> lx(n1), ly(n1), lz(n1);
    B.basis->values(ref[0], lx.data());
    B.basis->values(ref[1], ly.data());
    B.basis->values(ref[2], lz.data());
    int t = 0;
    for (int cc = 0; cc < n1; ++cc)
      for (int bb = 0; bb < n1; ++bb)
        for (int aa = 0; aa < n1; ++aa, ++t) {
          w[(size_t)r * maxn + t] = lx[aa] * ly[bb] * lz[cc];
          off[(size_t)r * maxn + t] = (long long)(e[2] * B.N + cc) * B.pz + (long long)(e[1] * B.N + bb) * B.py +
                                      (e[0] * B.N + aa);
        }
    dom[r] = found;
    nn[r] = t;
  }
  if ((size_t)R * maxn > c->recv_cap) {
    drop_graph(c);   // the captured kernels hold the old receiver buffers
    dfree(c->d_rw); dfree(c->d_roff); dfree(c->d_rdom); dfree(c->d_rnn);
    c->recv_cap = 0;
    int rc;
    if ((rc = dalloc(&c->d_rw, (size_t)R * maxn * sizeof(double))) ||
        (rc = dalloc(&c->d_roff, (size_t)R * maxn * sizeof(long long))) ||
        (rc = dalloc(&c->d_rdom, (size_t)R * maxn * sizeof(int))) ||
        (rc = dalloc(&c->d_rnn, (size_t)R * maxn * sizeof(int))))
      return rc;
    c->recv_cap = (size_t)R * maxn;
  }
  CUDA_TRY(cudaMemcpy(c->d_rw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_roff, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_rdom, dom.data(), R * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_rnn, nn.data(), R * sizeof(int), cudaMemcpyHostToDevice));
  return DGSEM_OK;
}

template <typename T>
int upload_field(dgsem_ctx* c, const std::vector<double>& h, void* const* dst, cudaStream_t s) {
  // h: [ndof] in node order; broadcast to every batch member, padded layout
  size_t off = 0;
  for (int d = 0; d < c->nd; ++d) {
    const Box& B = c->box[d];
    std::vector<T> tmp((size_t)B.bstride, T(0));
    for (int k = 0; k < B.L[2]; ++k)
      for (int j = 0; j < B.L[1]; ++j)
        for (int i = 0; i < B.L[0]; ++i)
          tmp[(size_t)k * B.pz + (size_t)j * B.py + i] = h.empty() ? T(0) : T(h[off + ((size_t)k * B.L[1] + j) * B.L[0] + i]);
    for (int b = 0; b < c->batch; ++b)
      CUDA_TRY(cudaMemcpyAsync(static_cast<T*>(dst[d]) + (size_t)b * B.bstride, tmp.data(), tmp.size() * sizeof(T),
                               cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    off += (size_t)B.L[0] * B.L[1] * B.L[2];
  }
  return DGSEM_OK;
}

// Per-run device views of the drive and trace buffers.
struct RunIO {
  const double* d_drive = nullptr;
  double* d_tr = nullptr;
  double* host_tr = nullptr;     // caller's host trace buffer (copied back at the end), or NULL
  size_t tr_n = 0;
  int R = 0;
  long long dbs = 0, dks = 0, tbs = 0, trs = 0;
  double* d_volt = nullptr;      // voltage record of this run (RX configured), or NULL
};

// Everything a run does before its time steps: tensor maps, status words,
// state reset or initial state, device copies of the drive, trace buffers.
template <typename T>
int run_prepare(dgsem_ctx* c, int nsteps, const double* drive, int R, double* traces_out, int flags, cudaStream_t s,
                RunIO& io) {
  int rc;
  if ((rc = refresh_tmaps(c))) return rc;
  CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
  const bool cont = (flags & DGSEM_RUN_CONTINUE) && c->state_valid;
  if (!cont) {
    if ((rc = zero_state(c, s))) return rc;
    if (c->has_init) {
      if ((rc = upload_field<T>(c, c->init_p, c->X, s))) return rc;
      if ((rc = upload_field<T>(c, c->init_v, c->V, s))) return rc;
      if ((rc = launch_step<T>(c, s, nullptr, 0, 0, 0, 0, nullptr, 0, 0, true))) return rc;
    }
    c->state_valid = true;
  }
  // drive: device copy if needed
  const size_t drive_n = (size_t)c->batch * c->K * nsteps;
  io.d_drive = nullptr;
  if (c->K > 0 && drive) {
    if (is_device_ptr(drive)) {
      io.d_drive = drive;
    } else {
      if (drive_n > c->drive_cap) {
        drop_graph(c);
        dfree(c->d_drive);
        if ((rc = dalloc(&c->d_drive, drive_n * sizeof(double)))) { c->drive_cap = 0; return rc; }
        c->drive_cap = drive_n;
      }
      CUDA_TRY(cudaMemcpyAsync(c->d_drive, drive, drive_n * sizeof(double), cudaMemcpyHostToDevice, s));
      io.d_drive = c->d_drive;
    }
  }
  io.R = R;
  io.tr_n = (size_t)c->batch * R * nsteps;
  io.host_tr = nullptr;
  io.d_tr = nullptr;
  if (R > 0) {
    if (is_device_ptr(traces_out)) {
      io.d_tr = traces_out;
    } else {
      io.host_tr = traces_out;
      if (io.tr_n > c->traces_cap) {
        drop_graph(c);
        dfree(c->d_traces);
        if ((rc = dalloc(&c->d_traces, io.tr_n * sizeof(double)))) { c->traces_cap = 0; return rc; }
        c->traces_cap = io.tr_n;
      }
      io.d_tr = c->d_traces;
    }
  }
  CUDA_TRY(cudaMemsetAsync(c->d_step, 0, sizeof(int), s));
  if (c->rx_switch >= 0 && c->K > 0) {
    if (!c->d_step_base && (rc = dalloc(&c->d_step_base, sizeof(long long)))) return rc;
    CUDA_TRY(cudaMemcpyAsync(c->d_step_base, &c->step, sizeof(long long), cudaMemcpyHostToDevice, s));
    const size_t vn = (size_t)c->batch * c->K * nsteps;
    if (vn > c->volt_cap) {
      drop_graph(c);   // the captured kernels hold the old buffer
      dfree(c->d_volt);
      if ((rc = dalloc(&c->d_volt, vn * sizeof(double)))) { c->volt_cap = 0; return rc; }
      c->volt_cap = vn;
    }
    io.d_volt = c->d_volt;
    c->volt_n = (long long)vn;
  } else {
    c->volt_n = 0;
  }
  io.dbs = (long long)c->K * nsteps;
  io.dks = nsteps;
  io.tbs = (long long)R * nsteps;
  io.trs = nsteps;
  return DGSEM_OK;
}

// Traces back to the host if needed, timings, device status word.
int run_finish(dgsem_ctx* c, int nsteps, const RunIO& io, cudaStream_t s) {
  c->step += nsteps;
  // divergence check: receiver traces (they sample p every step) and the PMUT state
  if (!c->d_nf) CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&c->d_nf), sizeof(int)));
  CUDA_TRY(cudaMemsetAsync(c->d_nf, 0, sizeof(int), s));
  CUDA_TRY(launch_nonfinite(io.d_tr, io.tr_n, c->d_nf, s));
  if (c->q_state) CUDA_TRY(launch_nonfinite(c->q_state, (size_t)3 * c->batch * c->K * c->M, c->d_nf, s));
  if (io.host_tr) CUDA_TRY(cudaMemcpyAsync(io.host_tr, io.d_tr, io.tr_n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  collect_timings(c);
  int err = 0, nf = 0;
  CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(&nf, c->d_nf, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    c->state_valid = false;
    return fail(DGSEM_ETIMEOUT, "a bounded device-side wait gave up (status %d); the state is invalid", err);
  }
  if (nf) {
    c->state_valid = false;
    return fail(DGSEM_EUNSTABLE, "non-finite receiver traces or PMUT state: the time step diverged (dt above the stability limit?)");
  }
  return DGSEM_OK;
}

// Stream and events of the second branch of a captured step.
int ensure_side(dgsem_ctx* c) {
  if (!c->side_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : c->fork_ev)
    if (!e) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return DGSEM_OK;
}

template <typename T>
int run_impl(dgsem_ctx* c, int nsteps, const double* drive, int R, double* traces_out, int flags, cudaStream_t s) {
  RunIO io;
  int rc = run_prepare<T>(c, nsteps, drive, R, traces_out, flags, s, io);
  if (rc) return rc;
  int done = 0;
  if (!c->profiling && nsteps >= 4) {
    // replay a captured block of G (even) steps; the kernels read the step
    // index from the device counter, so the same graph serves every block
    const int G = std::min(32, nsteps - (nsteps % 2));
    struct Key { int prec, batch, R, G; const void* dr; const void* tr; long long dbs, tbs; const void* x0; const void* y0; int t0, t1; } key;
    std::memset(&key, 0, sizeof(key));
    key.prec = c->prec; key.batch = c->batch; key.R = R; key.G = G; key.dr = io.d_drive; key.tr = io.d_tr;
    key.dbs = io.dbs; key.tbs = io.tbs; key.x0 = c->X[0]; key.y0 = c->Y[0];
    key.t0 = c->tile_pref[c->prec == DGSEM_FP32_MIXED ? 1 : 0][0]; key.t1 = c->tile_pref[c->prec == DGSEM_FP32_MIXED ? 1 : 0][1];
    std::vector<unsigned char> kb(reinterpret_cast<unsigned char*>(&key), reinterpret_cast<unsigned char*>(&key) + sizeof(key));
    if (!c->graph || c->graph_key != kb) {
      if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
      if (!c->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      if ((rc = ensure_side(c))) return rc;
      long long before[DGSEM_K_COUNT];
      for (int k = 0; k < DGSEM_K_COUNT; ++k) before[k] = c->launches[k];
      CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      int crc = DGSEM_OK;
      for (int n = 0; n < G && crc == DGSEM_OK; ++n)
        crc = launch_step<T>(c, c->cap_stream, io.d_drive, io.dbs, io.dks, 0, R, io.d_tr, io.tbs, io.trs, false,
                             c->side_stream, io.d_volt);
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
      if (crc) { if (g) cudaGraphDestroy(g); return crc; }
      if (ce != cudaSuccess) return fail(DGSEM_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) { c->graph = nullptr; return fail(DGSEM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce)); }
      for (int k = 0; k < DGSEM_K_COUNT; ++k) {
        c->graph_launches[k] = c->launches[k] - before[k];
        c->launches[k] = before[k];
      }
      c->graph_steps = G;
      c->graph_key = kb;
    }
    for (; done + G <= nsteps; done += G) {
      CUDA_TRY(cudaGraphLaunch(c->graph, s));
      for (int k = 0; k < DGSEM_K_COUNT; ++k) c->launches[k] += c->graph_launches[k];
    }
  }
  for (int n = done; n < nsteps; ++n) {
    rc = launch_step<T>(c, s, io.d_drive, io.dbs, io.dks, 0, R, io.d_tr, io.tbs, io.trs, false, nullptr, io.d_volt);
    if (rc) return rc;
  }
  return run_finish(c, nsteps, io, s);
}

// Several meshes in one launch: each context's block of G steps is captured
// on its own stream as a parallel branch of one CUDA graph, so uneven
// meshes (different sizes and orders) run concurrently.
template <typename T>
int run_multi_impl(int n, dgsem_ctx* const* ctxs, int nsteps, const double* const* drive, const int* n_recv,
                   double* const* traces, int flags, cudaStream_t s) {
  std::vector<RunIO> io(n);
  for (int i = 0; i < n; ++i) {
    int rc = run_prepare<T>(ctxs[i], nsteps, drive ? drive[i] : nullptr, n_recv ? n_recv[i] : 0,
                            traces ? traces[i] : nullptr, flags, s, io[i]);
    if (rc) return rc;
  }
  const int G = std::min(32, nsteps - (nsteps % 2));
  int done = 0;
  if (G >= 2) {
    cudaStream_t main = nullptr;
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    auto cleanup = [&]() {
      for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
      if (main) cudaStreamDestroy(main);
    };
    CUDA_TRY(cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking));
    for (auto& e : ev) {
      cudaError_t ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (ce != cudaSuccess) { cleanup(); return fail(DGSEM_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(ce)); }
    }
    for (int i = 0; i < n; ++i) {
      if (!ctxs[i]->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&ctxs[i]->cap_stream, cudaStreamNonBlocking));
      int rc = ensure_side(ctxs[i]);
      if (rc) { cleanup(); return rc; }
    }
    std::vector<std::array<long long, DGSEM_K_COUNT>> before(n), per(n);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < DGSEM_K_COUNT; ++k) before[i][k] = ctxs[i]->launches[k];
    cudaError_t ce = cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) { cleanup(); return fail(DGSEM_ECUDA, "graph capture: %s", cudaGetErrorString(ce)); }
    cudaEventRecord(ev[n], main);
    int crc = DGSEM_OK;
    for (int i = 0; i < n && crc == DGSEM_OK; ++i) {
      dgsem_ctx* c = ctxs[i];
      cudaStreamWaitEvent(c->cap_stream, ev[n], 0);
      for (int st = 0; st < G && crc == DGSEM_OK; ++st)
        crc = launch_step<T>(c, c->cap_stream, io[i].d_drive, io[i].dbs, io[i].dks, 0, io[i].R, io[i].d_tr, io[i].tbs,
                             io[i].trs, false, c->side_stream, io[i].d_volt);
      cudaEventRecord(ev[i], c->cap_stream);
      cudaStreamWaitEvent(main, ev[i], 0);
    }
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(main, &g);
    if (crc) { if (g) cudaGraphDestroy(g); cleanup(); return crc; }
    if (ce != cudaSuccess) { cleanup(); return fail(DGSEM_ECUDA, "graph capture: %s", cudaGetErrorString(ce)); }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { cleanup(); return fail(DGSEM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce)); }
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < DGSEM_K_COUNT; ++k) {
        per[i][k] = ctxs[i]->launches[k] - before[i][k];
        ctxs[i]->launches[k] = before[i][k];
      }
    for (; done + G <= nsteps; done += G) {
      ce = cudaGraphLaunch(exec, s);
      if (ce != cudaSuccess) break;
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < DGSEM_K_COUNT; ++k) ctxs[i]->launches[k] += per[i][k];
    }
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    cleanup();
    if (ce != cudaSuccess) return fail(DGSEM_ECUDA, "graph launch: %s", cudaGetErrorString(ce));
  }
  for (int st = done; st < nsteps; ++st)
    for (int i = 0; i < n; ++i) {
      int rc = launch_step<T>(ctxs[i], s, io[i].d_drive, io[i].dbs, io[i].dks, 0, io[i].R, io[i].d_tr, io[i].tbs,
                              io[i].trs, false, nullptr, io[i].d_volt);
      if (rc) return rc;
    }
  for (int i = 0; i < n; ++i) {
    int rc = run_finish(ctxs[i], nsteps, io[i], s);
    if (rc) return rc;
  }
  return DGSEM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* dgsem_last_error(void) { return g_err.c_str(); }
}  // extern "C"

int dg_fail_msg(int code, const char* msg) {
  g_err = msg;
  return code;
}

extern "C" {

int dgsem_mesh_create(const dgsem_mesh_desc* desc, dgsem_ctx** out) {
  if (!out) return fail(DGSEM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!desc || !desc->domains) return fail(DGSEM_EINVAL, "desc/domains is NULL");
  if (desc->ndomains < 1 || desc->ndomains > 2) return fail(DGSEM_EINVAL, "ndomains must be 1 or 2");
  for (int d = 0; d < desc->ndomains; ++d) {
    const dgsem_domain_desc& D = desc->domains[d];
    if (D.order < 1 || D.order > DG_MAXN) return fail(DGSEM_EINVAL, "domain %d: order %d not in [1, %d]", d, D.order, DG_MAXN);
    for (int k = 0; k < 3; ++k) {
      if (D.nelem[k] < 1) return fail(DGSEM_EINVAL, "domain %d: nelem[%d] < 1", d, k);
      if (!(D.extent[k] > 0.0) || !std::isfinite(D.extent[k])) return fail(DGSEM_EINVAL, "domain %d: extent[%d] <= 0", d, k);
      if ((long long)D.nelem[k] * D.order + 1 > (1 << 24)) return fail(DGSEM_EINVAL, "domain %d: lattice too large", d);
    }
    if (!(D.c > 0.0) || !(D.rho > 0.0)) return fail(DGSEM_EINVAL, "domain %d: c and rho must be > 0", d);
  }
  if (!(desc->dt > 0.0) && !(desc->cfl > 0.0)) return fail(DGSEM_EINVAL, "need dt > 0 or cfl > 0");
  if (desc->ndomains == 2 && !(desc->penalty_alpha > 0.0)) return fail(DGSEM_EINVAL, "penalty_alpha must be > 0");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  dgsem_ctx* c = new dgsem_ctx();
  c->device = dev;
  c->nd = desc->ndomains;
  c->alpha = desc->penalty_alpha;
  c->cfl = desc->cfl;
  double hmin = 1e300, cmax = 0.0;
  for (int d = 0; d < c->nd; ++d) {
    const dgsem_domain_desc& D = desc->domains[d];
    Box& B = c->box[d];
    c->basis[d] = new Basis1D(D.order);
    B.basis = c->basis[d];
    B.N = D.order;
    B.c = D.c;
    B.rho = D.rho;
    for (int k = 0; k < 3; ++k) {
      B.o[k] = D.origin[k];
      B.ext[k] = D.extent[k];
      B.ne[k] = D.nelem[k];
      B.h[k] = D.extent[k] / D.nelem[k];
      B.L[k] = D.nelem[k] * D.order + 1;
    }
    B.py = (int)round_up(B.L[0], 8);
    B.pz = (long long)B.py * B.L[1];
    B.bstride = round_up(B.pz * B.L[2], 64);
    double gap = 2.0;
    for (int i = 0; i < B.N; ++i) gap = std::min(gap, B.basis->x[i + 1] - B.basis->x[i]);
    for (int k = 0; k < 3; ++k) hmin = std::min(hmin, B.h[k] / 2.0 * gap);
    cmax = std::max(cmax, B.c);
    c->ndof += (long long)B.L[0] * B.L[1] * B.L[2];
    build_vol_spec(B, c->vspec[d]);
  }
  {
    int rc = dalloc(&c->d_err, sizeof(int));
    if (!rc) rc = dalloc(&c->d_step, sizeof(int));
    if (rc) { dgsem_destroy(c); return rc; }
    CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(c->d_step, 0, sizeof(int)));
  }
  c->dt = desc->dt > 0.0 ? desc->dt : desc->cfl * hmin / cmax;
  c->dt_cfl = c->dt;
  c->dt_fixed = desc->dt > 0.0;
  c->kappa = c->box[0].rho * c->box[0].c * c->box[0].c;
  if (c->nd == 2) {
    int rc = build_interface(c, desc);
    if (rc) { dgsem_destroy(c); return rc; }
  }
  // face lattice of Gamma_PMUT (primary z-min face)
  const Box& P = c->box[0];
  c->face_xy.resize((size_t)2 * P.L[0] * P.L[1]);
  for (int j = 0; j < P.L[1]; ++j)
    for (int i = 0; i < P.L[0]; ++i) {
      const int ex = std::min(i / P.N, P.ne[0] - 1), ax = i - ex * P.N;
      const int ey = std::min(j / P.N, P.ne[1] - 1), ay = j - ey * P.N;
      c->face_xy[2 * ((size_t)j * P.L[0] + i)] = P.o[0] + P.h[0] * (ex + 0.5 * (P.basis->x[ax] + 1.0));
      c->face_xy[2 * ((size_t)j * P.L[0] + i) + 1] = P.o[1] + P.h[1] * (ey + 0.5 * (P.basis->x[ay] + 1.0));
    }
  *out = c;
  return DGSEM_OK;
}

namespace {

// Largest damping rate C_ii/M_ii + alpha_i over the nodes of a box: the sum
// is separable (one term per axis), so its maximum is the sum of the axis
// maxima.
double box_damping_max(const Box& B, const double* abc, const std::vector<double>* zeta) {
  double tot = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    double m = 0.0;
    for (int i = 0; i < B.L[ax]; ++i) {
      double v = (zeta && !zeta[ax].empty()) ? zeta[ax][i] : 0.0;
      if (i == 0) v += abc[2 * ax];
      if (i == B.L[ax] - 1) v += abc[2 * ax + 1];
      m = std::max(m, v);
    }
    tot += m;
  }
  return tot;
}

// dt limit of the explicit damping terms: dt <= 1 / sigma over all boxes;
// box `box` takes the candidate abc / zeta.  Returns the new dt, or -1 if the
// caller fixed a dt above it.
double damped_dt(const dgsem_ctx* c, int box, const double* abc, const std::vector<double>* zeta) {
  double sigma = 0.0;
  for (int d = 0; d < c->nd; ++d)
    sigma = std::max(sigma, d == box ? box_damping_max(c->box[d], abc, zeta)
                                     : box_damping_max(c->box[d], c->vspec[d].abc, c->has_pml[d] ? c->zeta_h[d] : nullptr));
  double dt = c->dt_cfl;
  if (sigma > 0.0) dt = std::min(dt, 1.0 / sigma);
  if (c->dt_fixed && dt < c->dt_cfl) return -1.0;
  return dt;
}

// physical coordinate of lattice line i along axis ax of box B
double lattice_coord(const Box& B, int ax, int i) {
  const int e = std::min(i / B.N, B.ne[ax] - 1), a = i - e * B.N;
  return B.o[ax] + B.h[ax] * (e + 0.5 * (B.basis->x[a] + 1.0));
}

}  // namespace

int dgsem_set_absorbing(dgsem_ctx* c, int box, const int* sides) {
  if (!c || !sides) return fail(DGSEM_EINVAL, "NULL argument");
  if (box < 0 || box >= c->nd) return fail(DGSEM_EINVAL, "bad box %d", box);
  const Box& B = c->box[box];
  for (int s = 0; s < 6; ++s) {
    if (!sides[s]) continue;
    if (box == 0 && s == 4) return fail(DGSEM_EINVAL, "the primary z-min side carries Gamma_PMUT");
    if (c->nd == 2 && ((box == 0 && s == 5) || (box == 1 && s == 4)))
      return fail(DGSEM_EINVAL, "box %d side %d is the interface Gamma_I", box, s);
  }
  double abc[6];
  for (int s = 0; s < 6; ++s) abc[s] = sides[s] ? B.c * (2.0 / B.h[s / 2]) / B.basis->w[0] : 0.0;
  const double dt = damped_dt(c, box, abc, c->has_pml[box] ? c->zeta_h[box] : nullptr);
  if (dt < 0.0)
    return fail(DGSEM_EUNSTABLE, "dt = %.4e s exceeds the limit 1 / max(C/M + alpha) of the damping terms", c->dt_cfl);
  for (int s = 0; s < 6; ++s) c->vspec[box].abc[s] = abc[s];
  c->vspec[box].has_abc = 0;
  for (int s = 0; s < 6; ++s) c->vspec[box].has_abc |= sides[s] ? 1 : 0;
  c->dt = dt;
  // the captured step graph holds the old parameters, and the state's half-step
  // velocity belongs to the old dt
  drop_graph(c);
  c->state_valid = false;
  return DGSEM_OK;
}

int dgsem_set_pml(dgsem_ctx* c, int box, const double* thickness, double R) {
  if (!c || !thickness) return fail(DGSEM_EINVAL, "NULL argument");
  if (box < 0 || box >= c->nd) return fail(DGSEM_EINVAL, "bad box %d", box);
  const Box& B = c->box[box];
  bool any = false;
  for (int s = 0; s < 6; ++s) {
    if (!(thickness[s] >= 0.0) || !std::isfinite(thickness[s])) return fail(DGSEM_EINVAL, "thickness[%d] must be >= 0", s);
    if (thickness[s] == 0.0) continue;
    any = true;
    if (box == 0 && s == 4) return fail(DGSEM_EINVAL, "the primary z-min side carries Gamma_PMUT");
    if (c->nd == 2 && ((box == 0 && s == 5) || (box == 1 && s == 4)))
      return fail(DGSEM_EINVAL, "box %d side %d is the interface Gamma_I", box, s);
  }
  if (any && !(R > 0.0 && R < 1.0)) return fail(DGSEM_EINVAL, "R must lie in (0, 1)");
  int lo[3], hi[3];
  std::vector<double> zeta[3];
  for (int ax = 0; ax < 3; ++ax) {
    const double tl = thickness[2 * ax], th = thickness[2 * ax + 1];
    if (tl + th > B.ext[ax] * (1.0 + 1e-12)) return fail(DGSEM_EINVAL, "the layers of axis %d overlap", ax);
    lo[ax] = tl > 0.0 ? (int)std::ceil(tl / B.h[ax] - 1e-9) : 0;
    hi[ax] = th > 0.0 ? (int)std::ceil(th / B.h[ax] - 1e-9) : 0;
    zeta[ax].assign(B.L[ax], 0.0);
    const double x0 = B.o[ax], x1 = B.o[ax] + B.ext[ax];
    for (int i = 0; i < B.L[ax]; ++i) {
      const double x = lattice_coord(B, ax, i);
      for (int side = 0; side < 2; ++side) {
        const double t = side == 0 ? tl : th;
        if (t <= 0.0) continue;
        const double zt = B.c / t * std::log(1.0 / R);
        double sd = side == 0 ? (x0 + t - x) / t : (x - (x1 - t)) / t;
        sd = std::min(1.0, std::max(0.0, sd));
        zeta[ax][i] += zt * (sd - std::sin(2.0 * M_PI * sd) / (2.0 * M_PI));
      }
    }
  }
  const double dt = damped_dt(c, box, c->vspec[box].abc, any ? zeta : nullptr);
  if (dt < 0.0)
    return fail(DGSEM_EUNSTABLE, "dt = %.4e s exceeds the limit 1 / max(C/M + alpha) of the damping terms", c->dt_cfl);
  // layer elements: any axis index inside that axis' layers
  std::vector<int> slot((size_t)B.ne[0] * B.ne[1] * B.ne[2], -1), elem;
  if (any) {
    for (int ez = 0; ez < B.ne[2]; ++ez)
      for (int ey = 0; ey < B.ne[1]; ++ey)
        for (int ex = 0; ex < B.ne[0]; ++ex) {
          const bool in = ex < lo[0] || ex >= B.ne[0] - hi[0] || ey < lo[1] || ey >= B.ne[1] - hi[1] ||
                          ez < lo[2] || ez >= B.ne[2] - hi[2];
          if (!in) continue;
          const int el = ex + B.ne[0] * (ey + B.ne[1] * ez);
          slot[el] = (int)elem.size();
          elem.push_back(el);
        }
  }
  // replace the layer of this box
  free_run_state(c);
  dfree(c->d_pml_slot[box]); dfree(c->d_pml_elem[box]);
  for (int p = 0; p < 2; ++p)
    for (int ax = 0; ax < 3; ++ax) dfree(c->d_zeta[box][p][ax]);
  c->has_pml[box] = false;
  c->npml[box] = 0;
  for (int ax = 0; ax < 3; ++ax) c->zeta_h[box][ax].clear();
  c->dt = dt;
  c->state_valid = false;
  if (!any) return DGSEM_OK;
  int rc;
  if ((rc = upload(&c->d_pml_slot[box], slot)) || (rc = upload(&c->d_pml_elem[box], elem))) return rc;
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<float> zf(zeta[ax].begin(), zeta[ax].end());
    if ((rc = upload((double**)&c->d_zeta[box][0][ax], zeta[ax])) || (rc = upload((float**)&c->d_zeta[box][1][ax], zf)))
      return rc;
    c->zeta_h[box][ax] = zeta[ax];
    c->pml_lo[box][ax] = lo[ax];
    c->pml_hi[box][ax] = hi[ax];
  }
  c->npml[box] = (int)elem.size();
  c->has_pml[box] = true;
  return DGSEM_OK;
}

int dgsem_selftest_wait(dgsem_ctx* c, void* stream) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
  CUDA_TRY(launch_wait_probe(c->d_err, 1LL << 24, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
  if (err != 3) return fail(DGSEM_ECUDA, "the bounded wait did not report its give-up (status %d)", err);
  return DGSEM_OK;
}

int dgsem_get_dt(const dgsem_ctx* c, double* dt, double* dt_stable_max, long long* ndof) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (dt) *dt = c->dt;
  if (dt_stable_max) *dt_stable_max = c->dt_stable;
  if (ndof) *ndof = c->ndof;
  return DGSEM_OK;
}

int dgsem_pmut_nodes(const dgsem_ctx* c, int* n_nodes, const double** xy) {
  if (!c || !n_nodes || !xy) return fail(DGSEM_EINVAL, "NULL argument");
  *n_nodes = (int)(c->face_xy.size() / 2);
  *xy = c->face_xy.data();
  return DGSEM_OK;
}

int pmut_array_set(dgsem_ctx* c, int K, int M, const int* foot_ptr, const int* foot_node, const double* shape_un,
                   const double* freq_hz, const double* damping, const double* eta, const double* modal_mass) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (K < 0 || (K > 0 && (M < 1 || M > DG_MAXM))) return fail(DGSEM_EINVAL, "n_pmut %d / n_modes %d out of range", K, M);
  if (K > 0 && (!foot_ptr || !freq_hz || !damping || !eta)) return fail(DGSEM_EINVAL, "NULL PMUT array");
  const Box& P = c->box[0];
  const int nface = P.L[0] * P.L[1];
  int nnz = 0;
  if (K > 0) {
    if (foot_ptr[0] != 0) return fail(DGSEM_EINVAL, "foot_ptr[0] must be 0");
    for (int k = 0; k < K; ++k)
      if (foot_ptr[k + 1] < foot_ptr[k]) return fail(DGSEM_EINVAL, "foot_ptr not monotone at %d", k);
    nnz = foot_ptr[K];
    if (nnz > 0 && (!foot_node || !shape_un)) return fail(DGSEM_EINVAL, "NULL footprint arrays");
    for (int e = 0; e < nnz; ++e)
      if (foot_node[e] < 0 || foot_node[e] >= nface) return fail(DGSEM_EINVAL, "foot_node[%d] = %d out of range", e, foot_node[e]);
    for (int i = 0; i < K * M; ++i) {
      if (!(freq_hz[i] > 0.0) || !std::isfinite(freq_hz[i])) return fail(DGSEM_EINVAL, "freq_hz[%d] must be > 0", i);
      if (!(damping[i] >= 0.0) || !std::isfinite(damping[i])) return fail(DGSEM_EINVAL, "damping[%d] must be >= 0", i);
      if (!std::isfinite(eta[i])) return fail(DGSEM_EINVAL, "eta[%d] not finite", i);
      if (modal_mass && !(modal_mass[i] > 0.0)) return fail(DGSEM_EINVAL, "modal_mass[%d] must be > 0", i);
    }
    for (long long e = 0; e < (long long)nnz * M; ++e)
      if (!std::isfinite(shape_un[e])) return fail(DGSEM_EINVAL, "shape_un[%lld] not finite", e);
  }
  // release previous array (and any captured graph using it)
  drop_graph(c);
  dfree(c->d_fp_ptr); dfree(c->d_fp_off); dfree(c->d_Bm); dfree(c->d_Bm32); dfree(c->d_node_ptr); dfree(c->d_node_ent);
  dfree(c->d_ent_pmut); dfree(c->d_modal); dfree(c->q_state);
  dfree(c->d_rx_gain);
  c->rx_switch = -1;
  c->K = 0; c->M = 0; c->nnz = 0;
  c->state_valid = false;
  if (K == 0) return DGSEM_OK;
  // B_{j,km} = W_face(j) * U.n (GLL collocation of the membrane integrals)
  const Basis1D& bs = *P.basis;
  std::vector<int> h_fp_ptr(foot_ptr, foot_ptr + K + 1);
  std::vector<long long> h_off(nnz);
  std::vector<double> h_B((size_t)nnz * M);
  std::vector<int> ent_pmut(nnz);
  std::vector<int> node_cnt(nface + 1, 0);
  for (int k = 0; k < K; ++k)
    for (int e = foot_ptr[k]; e < foot_ptr[k + 1]; ++e) {
      const int node = foot_node[e];
      const int ix = node % P.L[0], iy = node / P.L[0];
      const double wf = P.h[0] * P.h[1] / 4.0 * bs.assembled_weight(ix, P.ne[0]) * bs.assembled_weight(iy, P.ne[1]);
      for (int m = 0; m < M; ++m) h_B[(size_t)e * M + m] = wf * shape_un[(size_t)e * M + m];
      h_off[e] = (long long)iy * P.py + ix;
      ent_pmut[e] = k;
      node_cnt[node + 1]++;
    }
  std::vector<int> node_ptr(nface + 1, 0);
  for (int i = 0; i < nface; ++i) node_ptr[i + 1] = node_ptr[i] + node_cnt[i + 1];
  std::vector<int> fill(node_ptr.begin(), node_ptr.end() - 1), node_ent(nnz);
  for (int e = 0; e < nnz; ++e) node_ent[fill[foot_node[e]]++] = e;
  std::vector<double> modal((size_t)4 * K * M);
  for (int i = 0; i < K * M; ++i) {
    const double om = 2.0 * M_PI * freq_hz[i];
    modal[i] = om * om;
    modal[(size_t)K * M + i] = 2.0 * damping[i] * om;
    modal[(size_t)2 * K * M + i] = modal_mass ? 1.0 / modal_mass[i] : 1.0;
    modal[(size_t)3 * K * M + i] = eta[i];
  }
  int rc;
  std::vector<float> h_B32(h_B.begin(), h_B.end());
  if ((rc = upload(&c->d_fp_ptr, h_fp_ptr)) || (rc = upload(&c->d_fp_off, h_off)) || (rc = upload(&c->d_Bm, h_B)) ||
      (rc = upload(&c->d_Bm32, h_B32)) ||
      (rc = upload(&c->d_node_ptr, node_ptr)) || (rc = upload(&c->d_node_ent, node_ent)) ||
      (rc = upload(&c->d_ent_pmut, ent_pmut)) || (rc = upload(&c->d_modal, modal)))
    return rc;
  c->K = K; c->M = M; c->nnz = nnz;
  // PMUT state buffers are sized with the run state
  free_run_state(c);
  return DGSEM_OK;
}

int pmut_set_receive(dgsem_ctx* c, long long n_switch, const double* capacitance, int sign) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  drop_graph(c);   // the captured PMUT launches hold the old switch
  if (n_switch < 0) {
    c->rx_switch = -1;
    return DGSEM_OK;
  }
  if (c->K == 0) return fail(DGSEM_ESTATE, "no PMUT array: call pmut_array_set first");
  if (!capacitance) return fail(DGSEM_EINVAL, "NULL capacitance");
  if (sign != 1 && sign != -1) return fail(DGSEM_EINVAL, "sign must be +1 or -1");
  std::vector<double> gain(c->K);
  for (int k = 0; k < c->K; ++k) {
    if (!(capacitance[k] > 0.0) || !std::isfinite(capacitance[k]))
      return fail(DGSEM_EINVAL, "capacitance[%d] must be > 0", k);
    gain[k] = sign / capacitance[k];
  }
  dfree(c->d_rx_gain);
  int rc = upload(&c->d_rx_gain, gain);
  if (rc) { c->rx_switch = -1; return rc; }
  c->rx_switch = n_switch;
  return DGSEM_OK;
}

int dgsem_get_voltages(const dgsem_ctx* c, double* out, size_t n) {
  if (!c || !out) return fail(DGSEM_EINVAL, "NULL argument");
  if (c->volt_n == 0 || !c->d_volt) return fail(DGSEM_ESTATE, "no voltage record: configure pmut_set_receive and run");
  if (n < (size_t)c->volt_n) return fail(DGSEM_EINVAL, "buffer of %zu doubles is smaller than %lld", n, c->volt_n);
  CUDA_TRY(cudaMemcpy(out, c->d_volt, (size_t)c->volt_n * sizeof(double), cudaMemcpyDeviceToHost));
  return DGSEM_OK;
}

int dgsem_set_state(dgsem_ctx* c, const double* p0, const double* v0) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  c->init_p.assign(p0 ? p0 : (const double*)nullptr, p0 ? p0 + c->ndof : (const double*)nullptr);
  c->init_v.assign(v0 ? v0 : (const double*)nullptr, v0 ? v0 + c->ndof : (const double*)nullptr);
  for (double x : c->init_p) if (!std::isfinite(x)) return fail(DGSEM_EINVAL, "p0 not finite");
  for (double x : c->init_v) if (!std::isfinite(x)) return fail(DGSEM_EINVAL, "v0 not finite");
  c->has_init = p0 || v0;
  c->state_valid = false;
  return DGSEM_OK;
}

int dgsem_run(dgsem_ctx* c, int precision, int batch, int nsteps, const double* drive, int n_recv,
              const double* recv_xyz, double* traces, int flags, void* stream) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return fail(DGSEM_EINVAL, "bad precision %d", precision);
  if (batch < 1 || nsteps < 0 || n_recv < 0) return fail(DGSEM_EINVAL, "batch >= 1, nsteps >= 0, n_recv >= 0 required");
  if (n_recv > 0 && (!recv_xyz || !traces)) return fail(DGSEM_EINVAL, "receivers need recv_xyz and traces");
  if (c->K > 0 && nsteps > 0 && !drive) return fail(DGSEM_EINVAL, "drive is NULL");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != c->device) return fail(DGSEM_EINVAL, "context belongs to device %d, current is %d", c->device, dev);
  if ((flags & DGSEM_RUN_CONTINUE) && (!c->state_valid || c->prec != precision || c->batch != batch))
    return fail(DGSEM_ESTATE, "DGSEM_RUN_CONTINUE needs a previous run with the same precision and batch");
  int rc = ensure_run_state(c, precision, batch);
  if (rc) return rc;
  if ((rc = setup_receivers(c, n_recv, recv_xyz))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a run that fails part-way leaves no state to continue from
  rc = precision == DGSEM_FP64 ? run_impl<double>(c, nsteps, drive, n_recv, traces, flags, s)
                               : run_impl<float>(c, nsteps, drive, n_recv, traces, flags, s);
  if (rc != DGSEM_OK) c->state_valid = false;
  return rc;
}

int dgsem_run_multi(int n, dgsem_ctx* const* ctxs, int precision, const int* batch, int nsteps,
                    const double* const* drive, const int* n_recv, const double* const* recv_xyz,
                    double* const* traces, int flags, void* stream) {
  if (n < 1 || !ctxs || !batch) return fail(DGSEM_EINVAL, "n >= 1, ctxs and batch are required");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return fail(DGSEM_EINVAL, "bad precision %d", precision);
  if (nsteps < 0) return fail(DGSEM_EINVAL, "nsteps < 0");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  for (int i = 0; i < n; ++i) {
    dgsem_ctx* c = ctxs[i];
    if (!c) return fail(DGSEM_EINVAL, "ctxs[%d] is NULL", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(DGSEM_EINVAL, "context %d appears twice", i);
    if (c->device != dev) return fail(DGSEM_EINVAL, "context %d belongs to device %d, current is %d", i, c->device, dev);
    if (batch[i] < 1) return fail(DGSEM_EINVAL, "batch[%d] < 1", i);
    const int R = n_recv ? n_recv[i] : 0;
    if (R < 0 || (R > 0 && (!recv_xyz || !recv_xyz[i] || !traces || !traces[i])))
      return fail(DGSEM_EINVAL, "context %d: receivers need recv_xyz and traces", i);
    if (c->K > 0 && nsteps > 0 && (!drive || !drive[i])) return fail(DGSEM_EINVAL, "context %d: drive is NULL", i);
    if ((flags & DGSEM_RUN_CONTINUE) && (!c->state_valid || c->prec != precision || c->batch != batch[i]))
      return fail(DGSEM_ESTATE, "context %d: DGSEM_RUN_CONTINUE needs a previous run with the same precision and batch", i);
    int rc = ensure_run_state(c, precision, batch[i]);
    if (rc) return rc;
    if ((rc = setup_receivers(c, R, R > 0 ? recv_xyz[i] : nullptr))) return rc;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = precision == DGSEM_FP64 ? run_multi_impl<double>(n, ctxs, nsteps, drive, n_recv, traces, flags, s)
                                         : run_multi_impl<float>(n, ctxs, nsteps, drive, n_recv, traces, flags, s);
  if (rc != DGSEM_OK)
    for (int i = 0; i < n; ++i) ctxs[i]->state_valid = false;
  return rc;
}

int dgsem_get_pressure(const dgsem_ctx* c, double* p, size_t len) {
  if (!c || !p) return fail(DGSEM_EINVAL, "NULL argument");
  if (!c->X[0] || !c->state_valid) return fail(DGSEM_ESTATE, "no state: call dgsem_run first");
  if (len < (size_t)c->batch * c->ndof) return fail(DGSEM_EINVAL, "len %zu < batch*ndof", len);
  CUDA_TRY(cudaDeviceSynchronize());
  const size_t es = elem_size(c->prec);
  size_t off = 0;
  for (int b = 0; b < c->batch; ++b)
    for (int d = 0; d < c->nd; ++d) {
      const Box& B = c->box[d];
      std::vector<unsigned char> tmp((size_t)B.bstride * es);
      CUDA_TRY(cudaMemcpy(tmp.data(), static_cast<const unsigned char*>(c->X[d]) + (size_t)b * B.bstride * es,
                          tmp.size(), cudaMemcpyDeviceToHost));
      for (int k = 0; k < B.L[2]; ++k)
        for (int j = 0; j < B.L[1]; ++j)
          for (int i = 0; i < B.L[0]; ++i) {
            const size_t g = (size_t)k * B.pz + (size_t)j * B.py + i;
            p[off++] = es == 8 ? reinterpret_cast<const double*>(tmp.data())[g]
                               : (double)reinterpret_cast<const float*>(tmp.data())[g];
          }
    }
  return DGSEM_OK;
}

// checkpoint layout: header | X, Y, V of each box | q, q', q''
struct CkptHeader {
  char magic[8];
  int prec, batch, nd, K, M;
  long long step, ndof, bstride[2];
};

int dgsem_state_save(const dgsem_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return fail(DGSEM_EINVAL, "NULL argument");
  if (!c->state_valid) return fail(DGSEM_ESTATE, "no state to save");
  if (c->has_pml[0] || c->has_pml[1]) return fail(DGSEM_ESTATE, "checkpoints of a state with a PML are not supported");
  const size_t es = elem_size(c->prec);
  size_t need = sizeof(CkptHeader);
  for (int d = 0; d < c->nd; ++d) need += 3 * (size_t)c->batch * c->box[d].bstride * es;
  need += (size_t)3 * c->batch * c->K * c->M * sizeof(double);
  if (!buf) { *len = need; return DGSEM_OK; }
  if (*len < need) return fail(DGSEM_EINVAL, "buffer too small (%zu < %zu)", *len, need);
  CUDA_TRY(cudaDeviceSynchronize());
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "DGSEMCK1", 8);
  h.prec = c->prec; h.batch = c->batch; h.nd = c->nd; h.K = c->K; h.M = c->M;
  h.step = c->step; h.ndof = c->ndof;
  for (int d = 0; d < c->nd; ++d) h.bstride[d] = c->box[d].bstride;
  unsigned char* o = static_cast<unsigned char*>(buf);
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  for (int d = 0; d < c->nd; ++d) {
    const size_t bytes = (size_t)c->batch * c->box[d].bstride * es;
    for (void* src : {c->X[d], c->Y[d], c->V[d]}) {
      CUDA_TRY(cudaMemcpy(o, src, bytes, cudaMemcpyDeviceToHost));
      o += bytes;
    }
  }
  const size_t qb = (size_t)3 * c->batch * c->K * c->M * sizeof(double);
  if (qb) CUDA_TRY(cudaMemcpy(o, c->q_state, qb, cudaMemcpyDeviceToHost));
  *len = need;
  return DGSEM_OK;
}

int dgsem_state_load(dgsem_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) return fail(DGSEM_EINVAL, "NULL argument");
  if (len < sizeof(CkptHeader)) return fail(DGSEM_EINVAL, "buffer too small");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, "DGSEMCK1", 8) != 0) return fail(DGSEM_EINVAL, "not a dgsem checkpoint");
  if (h.nd != c->nd || h.K != c->K || h.M != c->M || h.ndof != c->ndof)
    return fail(DGSEM_EINVAL, "checkpoint does not match this mesh / PMUT array");
  for (int d = 0; d < c->nd; ++d)
    if (h.bstride[d] != c->box[d].bstride) return fail(DGSEM_EINVAL, "checkpoint layout mismatch");
  if (h.batch < 1 || (h.prec != DGSEM_FP64 && h.prec != DGSEM_FP32_MIXED)) return fail(DGSEM_EINVAL, "bad checkpoint header");
  const size_t es = elem_size(h.prec);
  size_t need = sizeof(CkptHeader);
  for (int d = 0; d < c->nd; ++d) need += 3 * (size_t)h.batch * c->box[d].bstride * es;
  need += (size_t)3 * h.batch * c->K * c->M * sizeof(double);
  if (len < need) return fail(DGSEM_EINVAL, "checkpoint truncated (%zu < %zu)", len, need);
  int rc = ensure_run_state(c, h.prec, h.batch);
  if (rc) return rc;
  const unsigned char* o = static_cast<const unsigned char*>(buf) + sizeof(h);
  for (int d = 0; d < c->nd; ++d) {
    const size_t bytes = (size_t)h.batch * c->box[d].bstride * es;
    for (void* dst : {c->X[d], c->Y[d], c->V[d]}) {
      CUDA_TRY(cudaMemcpy(dst, o, bytes, cudaMemcpyHostToDevice));
      o += bytes;
    }
  }
  const size_t qb = (size_t)3 * h.batch * c->K * c->M * sizeof(double);
  if (qb) CUDA_TRY(cudaMemcpy(c->q_state, o, qb, cudaMemcpyHostToDevice));
  c->step = h.step;
  c->state_valid = true;
  c->has_init = false;
  return DGSEM_OK;
}

int dgsem_energy(dgsem_ctx* c, double* e, int n) {
  if (!c || !e) return fail(DGSEM_EINVAL, "NULL argument");
  if (!c->state_valid) return fail(DGSEM_ESTATE, "no state: run first");
  if (n < c->batch) return fail(DGSEM_EINVAL, "e holds %d values, %d needed", n, c->batch);
  const bool f32 = c->prec == DGSEM_FP32_MIXED;
  int rc = refresh_tmaps(c);
  if (rc) return rc;
  cudaStream_t s = 0;
  std::vector<void*> tmp;
  auto cleanup = [&]() { for (void* p : tmp) cudaFree(p); };
  // The operator is applied in FP64 to p^{n+1}: the state's own buffer in
  // FP64, an FP64 copy of it (with its own tensor map and FP64 interface
  // buffers) for an FP32 state.  W = -M^-1 K p^{n+1} (volume kernel with
  // v = 0, dtv = 1, dtp = 0, no forcing, absorbing or layer terms); P2
  // receives the unchanged p_out.
  double* W[2] = {nullptr, nullptr};
  double* P2[2] = {nullptr, nullptr};
  double* Y64[2] = {nullptr, nullptr};
  double* Ra64[2] = {nullptr, nullptr};
  double* Rb64[2] = {nullptr, nullptr};
  double* Ga64[2] = {nullptr, nullptr};
  double* Gb64[2] = {nullptr, nullptr};
  CUtensorMap tm64[2];
  double* w1[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  double* d_red = nullptr;
  if ((rc = dalloc(&d_red, 2 * sizeof(double) * c->batch))) return rc;
  tmp.push_back(d_red);
  for (int d = 0; d < c->nd; ++d) {
    const Box& B = c->box[d];
    const size_t cnt = (size_t)c->batch * B.bstride;
    const size_t bytes = cnt * sizeof(double);
    if ((rc = dalloc(&W[d], bytes)) || (rc = dalloc(&P2[d], bytes))) { cleanup(); return rc; }
    tmp.push_back(W[d]);
    tmp.push_back(P2[d]);
    CUDA_TRY(cudaMemsetAsync(W[d], 0, bytes, s));
    if (f32) {
      if ((rc = dalloc(&Y64[d], bytes))) { cleanup(); return rc; }
      tmp.push_back(Y64[d]);
      CUDA_TRY(launch_widen(static_cast<const float*>(c->Y[d]), Y64[d], (long long)cnt, s));
      unsigned box[3], vbox[3];
      if (!vol_tma_box_f64(B.N, c->tile_pref[0][d], box, vbox)) { cleanup(); return fail(DGSEM_EINVAL, "no FP64 tile variant"); }
      if ((rc = make_tmap(&tm64[d], Y64[d], B, c->batch, DGSEM_FP64, box))) { cleanup(); return rc; }
      if (c->has_iface) {
        const size_t rb = (size_t)c->batch * B.ne[0] * B.ne[1] * (B.N + 1) * (B.N + 1) * sizeof(double);
        const size_t gb = (size_t)c->batch * B.L[1] * B.py * sizeof(double);
        if ((rc = dalloc(&Ra64[d], rb)) || (rc = dalloc(&Rb64[d], rb)) || (rc = dalloc(&Ga64[d], gb)) ||
            (rc = dalloc(&Gb64[d], gb))) {
          for (double* q : {Ra64[d], Rb64[d], Ga64[d], Gb64[d]}) if (q) tmp.push_back(q);
          cleanup();
          return rc;
        }
        for (double* q : {Ra64[d], Rb64[d], Ga64[d], Gb64[d]}) tmp.push_back(q);
        CUDA_TRY(cudaMemsetAsync(Ga64[d], 0, gb, s));
        CUDA_TRY(cudaMemsetAsync(Gb64[d], 0, gb, s));
      }
    } else {
      Y64[d] = static_cast<double*>(c->Y[d]);
      tm64[d] = c->tmap_y[d];
      Ra64[d] = static_cast<double*>(c->Ra[d]); Rb64[d] = static_cast<double*>(c->Rb[d]);
      Ga64[d] = static_cast<double*>(c->Ga[d]); Gb64[d] = static_cast<double*>(c->Gb[d]);
    }
    for (int k = 0; k < 3; ++k) {
      std::vector<double> w(B.L[k]);
      for (int i = 0; i < B.L[k]; ++i) w[i] = B.basis->assembled_weight(i, B.ne[k]);
      if ((rc = upload(&w1[d][k], w))) { cleanup(); return rc; }
      tmp.push_back(w1[d][k]);
    }
  }
  CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
  if (c->has_iface) {
    IfaceArgs<double> a = iface_args<double>(c);
    a.pp = Y64[0];
    a.ps = Y64[1];
    a.Rap = Ra64[0]; a.Rbp = Rb64[0]; a.Ras = Ra64[1]; a.Rbs = Rb64[1];
    CUDA_TRY(launch_iface<double>(a, c->batch, s));
    for (int d = 0; d < c->nd; ++d) {
      const Box& B = c->box[d];
      FaceAsmArgs<double> f;
      f.Ra = Ra64[d]; f.Rb = Rb64[d]; f.ga = Ga64[d]; f.gb = Gb64[d];
      f.N = B.N; f.ne0 = B.ne[0]; f.ne1 = B.ne[1]; f.L0 = B.L[0]; f.L1 = B.L[1]; f.py = B.py;
      f.rbs = (long long)B.ne[0] * B.ne[1] * (B.N + 1) * (B.N + 1);
      f.gbs = (long long)B.L[1] * B.py;
      CUDA_TRY(launch_face_asm<double>(f, c->batch, s));
    }
  }
  for (int d = 0; d < c->nd; ++d) {
    VolSpec v = c->vspec[d];
    v.has_abc = 0;
    v.has_pml = 0;
    v.has_pmut = 0;
    v.tmap = &tm64[d];
    v.tmap_v = nullptr;
    v.err = c->d_err;
    v.tile = c->tile_pref[0][d];
    v.step = nullptr;
    v.shape_out = nullptr;
    v.p_in = Y64[d]; v.p_out = P2[d]; v.v = W[d];
    v.dtv = 1.0; v.dtp = 0.0;
    v.ga = Ga64[d]; v.gb = Gb64[d];
    v.gbs = (long long)c->box[d].L[1] * c->box[d].py;
    CUDA_TRY(launch_vol<double>(v, c->batch, s));
  }
  // e_b = 1/2 v.M v + 1/2 p^n.K p^{n+1} = 1/2 (v.M v - p^n.M W)
  CUDA_TRY(cudaMemsetAsync(d_red, 0, 2 * sizeof(double) * c->batch, s));
  for (int b = 0; b < c->batch; ++b)
    for (int d = 0; d < c->nd; ++d) {
      const Box& B = c->box[d];
      const long long o = (long long)b * B.bstride;
      const double scale = B.h[0] * B.h[1] * B.h[2] / 8.0;
      if (f32) {
        const float* V = static_cast<const float*>(c->V[d]) + o;
        const float* X = static_cast<const float*>(c->X[d]) + o;
        // v.M v: v widened into P2, which the volume launch no longer needs
        CUDA_TRY(launch_widen(V, P2[d] + o, B.bstride, s));
        CUDA_TRY(launch_mdot(V, P2[d] + o, w1[d][0], w1[d][1], w1[d][2], B.L[0], B.L[1], B.L[2], B.py, B.pz, scale,
                             d_red + 2 * b, s));
        CUDA_TRY(launch_mdot(X, W[d] + o, w1[d][0], w1[d][1], w1[d][2], B.L[0], B.L[1], B.L[2], B.py, B.pz, scale,
                             d_red + 2 * b + 1, s));
      } else {
        const double* V = static_cast<const double*>(c->V[d]) + o;
        const double* X = static_cast<const double*>(c->X[d]) + o;
        CUDA_TRY(launch_mdot(V, V, w1[d][0], w1[d][1], w1[d][2], B.L[0], B.L[1], B.L[2], B.py, B.pz, scale,
                             d_red + 2 * b, s));
        CUDA_TRY(launch_mdot(X, W[d] + o, w1[d][0], w1[d][1], w1[d][2], B.L[0], B.L[1], B.L[2], B.py, B.pz, scale,
                             d_red + 2 * b + 1, s));
      }
    }
  std::vector<double> red(2 * (size_t)c->batch);
  CUDA_TRY(cudaMemcpy(red.data(), d_red, red.size() * sizeof(double), cudaMemcpyDeviceToHost));
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  cleanup();
  if (err) return fail(DGSEM_ETIMEOUT, "a bounded device-side wait gave up during the energy diagnostic");
  for (int b = 0; b < c->batch; ++b) e[b] = 0.5 * (red[2 * b] - red[2 * b + 1]);
  return DGSEM_OK;
}

int dgsem_get_pmut_state(const dgsem_ctx* c, double* q, double* qd, double* qdd, size_t n) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (!c->state_valid) return fail(DGSEM_ESTATE, "no state: run first");
  if (c->K == 0 || !c->q_state) return fail(DGSEM_ESTATE, "no PMUT array");
  const size_t km = (size_t)c->batch * c->K * c->M;
  if (n < km) return fail(DGSEM_EINVAL, "arrays hold %zu values, [batch][n_pmut][n_modes] = %zu needed", n, km);
  CUDA_TRY(cudaDeviceSynchronize());
  double* dst[3] = {q, qd, qdd};
  for (int i = 0; i < 3; ++i)
    if (dst[i]) CUDA_TRY(cudaMemcpy(dst[i], c->q_state + i * km, km * sizeof(double), cudaMemcpyDeviceToHost));
  return DGSEM_OK;
}

int dgsem_check_stability(dgsem_ctx* c, int iters, double* lambda_max) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (iters < 1) return fail(DGSEM_EINVAL, "iters must be >= 1");
  if (lambda_max) *lambda_max = 0.0;
  int rc = ensure_run_state(c, DGSEM_FP64, 1);
  if (rc) return rc;
  if ((rc = refresh_tmaps(c))) return rc;
  cudaStream_t s = 0;
  if ((rc = zero_state(c, s))) return rc;
  c->state_valid = false;
  CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
  // assembled 1D GLL weights of every box (the lumped mass is their product)
  std::vector<double*> dw;
  auto cleanup = [&]() { for (double* p : dw) cudaFree(p); };
  double* d_red = nullptr;
  if ((rc = dalloc(&d_red, 2 * sizeof(double)))) return rc;
  dw.push_back(d_red);
  double* w1[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  for (int d = 0; d < c->nd; ++d)
    for (int k = 0; k < 3; ++k) {
      std::vector<double> w(c->box[d].L[k]);
      for (int i = 0; i < c->box[d].L[k]; ++i) w[i] = c->box[d].basis->assembled_weight(i, c->box[d].ne[k]);
      if ((rc = upload(&w1[d][k], w))) { cleanup(); return rc; }
      dw.push_back(w1[d][k]);
    }
  // deterministic pseudo-random start vector (LCG)
  std::vector<double> x0(c->ndof);
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  for (auto& v : x0) { st = st * 6364136223846793005ull + 1442695040888963407ull; v = (double)(st >> 11) / 9007199254740992.0 - 0.5; }
  if ((rc = upload_field<double>(c, x0, c->X, s))) { cleanup(); return rc; }
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    // V = -M^-1 K X  (volume kernel with v = 0, dtv = 1, dtp = 0, no PMUT forcing)
    for (int d = 0; d < c->nd; ++d) CUDA_TRY(cudaMemsetAsync(c->V[d], 0, c->box[d].bstride * sizeof(double), s));
    if (c->has_iface) {
      IfaceArgs<double> a = iface_args<double>(c);
      a.pp = static_cast<const double*>(c->X[0]);
      a.ps = static_cast<const double*>(c->X[1]);
      CUDA_TRY(launch_iface<double>(a, 1, s));
      if ((rc = launch_face_assembly<double>(c, s, 1, false))) { cleanup(); return rc; }
    }
    for (int d = 0; d < c->nd; ++d) {
      VolSpec v = c->vspec[d];
      v.has_abc = 0;     // M^-1 K only (v = 0 makes the damping terms vanish anyway)
      v.has_pml = 0;
      v.tmap = &c->tmap_x[d];
      v.tmap_v = c->has_tmap_v[d] ? &c->tmap_v[d] : nullptr;
      v.err = c->d_err;
      v.tile = c->tile_pref[0][d];
      v.p_in = c->X[d]; v.p_out = c->Y[d]; v.v = c->V[d];
      v.dtv = 1.0; v.dtp = 0.0;
      v.ga = c->Ga[d]; v.gb = c->Gb[d];
      v.gbs = (long long)c->box[d].L[1] * c->box[d].py;
      CUDA_TRY(launch_vol<double>(v, 1, s));
    }
    // Rayleigh quotient x.K x / x.M x = -(x.M v)/(x.M x), and the norm of v
    CUDA_TRY(cudaMemsetAsync(d_red, 0, 2 * sizeof(double), s));
    for (int d = 0; d < c->nd; ++d) {
      const Box& B = c->box[d];
      const double scale = B.h[0] * B.h[1] * B.h[2] / 8.0;
      CUDA_TRY(launch_mdot((const double*)c->X[d], (const double*)c->V[d], w1[d][0], w1[d][1], w1[d][2], B.L[0], B.L[1],
                           B.L[2], B.py, B.pz, scale, d_red, s));
      CUDA_TRY(launch_mdot((const double*)c->V[d], (const double*)c->V[d], w1[d][0], w1[d][1], w1[d][2], B.L[0], B.L[1],
                           B.L[2], B.py, B.pz, scale, d_red + 1, s));
    }
    double red[2];
    CUDA_TRY(cudaMemcpy(red, d_red, sizeof(red), cudaMemcpyDeviceToHost));
    // x is M-normalised (x.M x = 1) after the first iteration
    double xmx = 1.0;
    if (it == 0) {
      CUDA_TRY(cudaMemsetAsync(d_red, 0, sizeof(double), s));
      for (int d = 0; d < c->nd; ++d) {
        const Box& B = c->box[d];
        CUDA_TRY(launch_mdot((const double*)c->X[d], (const double*)c->X[d], w1[d][0], w1[d][1], w1[d][2], B.L[0],
                             B.L[1], B.L[2], B.py, B.pz, B.h[0] * B.h[1] * B.h[2] / 8.0, d_red, s));
      }
      CUDA_TRY(cudaMemcpy(&xmx, d_red, sizeof(double), cudaMemcpyDeviceToHost));
    }
    lam = -red[0] / xmx;
    if (!(red[1] > 0.0) || !std::isfinite(red[1])) break;
    const double inv = 1.0 / std::sqrt(red[1]);
    for (int d = 0; d < c->nd; ++d)
      CUDA_TRY(launch_scale((double*)c->X[d], (const double*)c->V[d], inv, c->box[d].bstride, s));
  }
  CUDA_TRY(cudaDeviceSynchronize());
  cleanup();
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return fail(DGSEM_ETIMEOUT, "a bounded device-side wait gave up during the stability check");
  if (lambda_max) *lambda_max = lam;
  if (!(lam > 0.0)) return fail(DGSEM_EUNSTABLE, "lambda_max estimate %g is not positive", lam);
  c->dt_stable = 2.0 / std::sqrt(lam);
  if (c->dt > 0.95 * c->dt_stable)
    return fail(DGSEM_EUNSTABLE, "dt = %.4e s exceeds 0.95 * 2/sqrt(lambda_max) = %.4e s", c->dt, 0.95 * c->dt_stable);
  return DGSEM_OK;
}

int dgsem_set_tiles(dgsem_ctx* c, int precision, const int* tiles) {
  if (!c || !tiles) return fail(DGSEM_EINVAL, "NULL argument");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return fail(DGSEM_EINVAL, "bad precision");
  for (int d = 0; d < c->nd; ++d) {
    unsigned box[3], vbox[3];
    const int nv = precision == DGSEM_FP32_MIXED ? vol_tma_box_f32(c->box[d].N, tiles[d], box, vbox)
                                                 : vol_tma_box_f64(c->box[d].N, tiles[d], box, vbox);
    if (!nv) return fail(DGSEM_EINVAL, "box %d: no tile variant %d for order %d", d, tiles[d], c->box[d].N);
  }
  for (int d = 0; d < c->nd; ++d) c->tile_pref[precision == DGSEM_FP32_MIXED ? 1 : 0][d] = tiles[d];
  return DGSEM_OK;
}

int dgsem_set_layers(dgsem_ctx* c, const int* layers_per_cta) {
  if (!c || !layers_per_cta) return fail(DGSEM_EINVAL, "NULL argument");
  for (int d = 0; d < c->nd; ++d)
    if (layers_per_cta[d] < 0) return fail(DGSEM_EINVAL, "box %d: layers_per_cta %d < 0", d, layers_per_cta[d]);
  for (int d = 0; d < c->nd; ++d) c->vspec[d].layers_per_cta = std::min(layers_per_cta[d], c->box[d].ne[2]);
  drop_graph(c);   // the captured launches hold the old grid
  return DGSEM_OK;
}

int dgsem_vol_launch(const dgsem_ctx* c, int box, int* shape) {
  if (!c || !shape) return fail(DGSEM_EINVAL, "NULL argument");
  if (box < 0 || box >= c->nd) return fail(DGSEM_EINVAL, "box %d out of range", box);
  if (c->vol_shape[box][0] == 0) return fail(DGSEM_ESTATE, "no volume launch of box %d yet", box);
  for (int i = 0; i < 8; ++i) shape[i] = c->vol_shape[box][i];
  return DGSEM_OK;
}

int dgsem_num_tiles(const dgsem_ctx* c, int precision, int box, int* n) {
  if (!c || !n) return fail(DGSEM_EINVAL, "NULL argument");
  if (box < 0 || box >= c->nd) return fail(DGSEM_EINVAL, "bad box %d", box);
  unsigned b3[3], v3[3];
  *n = precision == DGSEM_FP32_MIXED ? vol_tma_box_f32(c->box[box].N, 0, b3, v3)
                                     : vol_tma_box_f64(c->box[box].N, 0, b3, v3);
  return DGSEM_OK;
}

int dgsem_autotune(dgsem_ctx* c, int precision, int batch, int reps, int* chosen, void* stream) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return fail(DGSEM_EINVAL, "bad precision");
  if (batch < 1 || reps < 1) return fail(DGSEM_EINVAL, "batch and reps must be >= 1");
  int rc = ensure_run_state(c, precision, batch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = zero_state(c, s))) return rc;
  CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
  const int pi = precision == DGSEM_FP32_MIXED ? 1 : 0;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  for (int d = 0; d < c->nd; ++d) {
    unsigned b3[3], v3[3];
    const int nv = pi ? vol_tma_box_f32(c->box[d].N, 0, b3, v3) : vol_tma_box_f64(c->box[d].N, 0, b3, v3);
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < nv; ++v) {
      c->tile_pref[pi][d] = v;
      if ((rc = refresh_tmaps(c))) break;
      VolSpec sp = c->vspec[d];
      sp.tmap = &c->tmap_y[d];
      sp.tmap_v = c->has_tmap_v[d] ? &c->tmap_v[d] : nullptr;
      sp.tmap_pst = c->has_tmap_v[d] ? &c->tmap_px[d] : nullptr;
      sp.err = c->d_err;
      sp.tile = v;
      sp.p_in = c->Y[d]; sp.p_out = c->X[d]; sp.v = c->V[d];
      sp.dtv = c->dt; sp.dtp = c->dt;
      sp.ga = c->Ga[d]; sp.gb = c->Gb[d];
      sp.gbs = (long long)c->box[d].L[1] * c->box[d].py;
      sp.has_abc = 0;
      sp.has_pml = 0;
      cudaError_t e = pi ? launch_vol<float>(sp, batch, s) : launch_vol<double>(sp, batch, s);   // warm-up
      if (e != cudaSuccess) { cudaGetLastError(); continue; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) e = pi ? launch_vol<float>(sp, batch, s) : launch_vol<double>(sp, batch, s);
      cudaEventRecord(e1, s);
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); continue; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = v; }
    }
    c->tile_pref[pi][d] = best;
    if (chosen) chosen[d] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->state_valid = false;
  if (rc) return rc;
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return fail(DGSEM_ETIMEOUT, "a bounded device-side wait gave up during autotuning");
  return refresh_tmaps(c);
}

int dgsem_profile(dgsem_ctx* c, int enable) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  c->profiling = enable != 0;
  for (int k = 0; k < DGSEM_K_COUNT; ++k) { c->kernel_ms[k] = 0.0; c->launches[k] = 0; }
  c->ev_used.clear();
  return DGSEM_OK;
}

int dgsem_kernel_stats(const dgsem_ctx* c, int kind, double* total_ms, long long* launches) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (kind < 0 || kind >= DGSEM_K_COUNT) return fail(DGSEM_EINVAL, "bad kernel kind %d", kind);
  if (total_ms) *total_ms = c->kernel_ms[kind];
  if (launches) *launches = c->launches[kind];
  return DGSEM_OK;
}

void dgsem_destroy(dgsem_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  free_run_state(c);
  dfree(c->d_cf_col); dfree(c->d_cf_ptr); dfree(c->d_ff_col); dfree(c->d_ff_sx); dfree(c->d_ff_sy);
  dfree(c->d_tab[0]); dfree(c->d_tab[1]);
  dfree(c->d_fp_ptr); dfree(c->d_fp_off); dfree(c->d_Bm); dfree(c->d_Bm32); dfree(c->d_node_ptr); dfree(c->d_node_ent);
  dfree(c->d_ent_pmut); dfree(c->d_modal);
  dfree(c->d_drive); dfree(c->d_traces);
  dfree(c->d_rw); dfree(c->d_roff); dfree(c->d_rdom); dfree(c->d_rnn);
  dfree(c->d_err); dfree(c->d_nf);
  dfree(c->d_step);
  dfree(c->d_rx_gain); dfree(c->d_step_base); dfree(c->d_volt);
  for (int d = 0; d < 2; ++d) {
    dfree(c->d_pml_slot[d]); dfree(c->d_pml_elem[d]);
    for (int p = 0; p < 2; ++p)
      for (int ax = 0; ax < 3; ++ax) dfree(c->d_zeta[d][p][ax]);
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  for (cudaEvent_t e : c->fork_ev)
    if (e) cudaEventDestroy(e);
  delete c->basis[0];
  delete c->basis[1];
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Receiver sampling without device allocation.
//
// dgsem_sample_noalloc keeps its receiver table (containing element, tensor
// Lagrange weights and node offsets of up to NA_MAX_RECV points) in the
// file-scope device array below instead of buffers from cudaMalloc, then runs
// the receiver-sampling kernel of the time loop on it.  The array lives for
// the lifetime of the library on every device that loads it.
// ---------------------------------------------------------------------------
namespace {

constexpr int NA_MAX_RECV = 64;                                   // receivers per call
constexpr int NA_MAX_NODES = (DG_MAXN + 1) * (DG_MAXN + 1) * (DG_MAXN + 1);
constexpr size_t NA_OFF_STATUS = 0;                               // int status word
constexpr size_t NA_OFF_XYZ = 256;                                // [R][3] double
constexpr size_t NA_OFF_W = NA_OFF_XYZ + (((size_t)NA_MAX_RECV * 3 * sizeof(double) + 255) / 256) * 256;
constexpr size_t NA_OFF_OFF = NA_OFF_W + (size_t)NA_MAX_RECV * NA_MAX_NODES * sizeof(double);
constexpr size_t NA_OFF_DOM = NA_OFF_OFF + (size_t)NA_MAX_RECV * NA_MAX_NODES * sizeof(long long);
constexpr size_t NA_OFF_NN = NA_OFF_DOM + (size_t)NA_MAX_RECV * sizeof(int);
constexpr size_t NA_BYTES = NA_OFF_NN + (size_t)NA_MAX_RECV * sizeof(int);   // about 0.75 MiB

static __device__ __align__(256) unsigned char g_sample_scratch[NA_BYTES];

// device address of g_sample_scratch, looked up once per device (under the
// mutex: host threads may make their first calls concurrently).  The address
// is not refreshed after cudaDeviceReset.
constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_sample_scratch_addr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_sample_scratch_mu;

struct NaBox {
  double o[3], h[3], ext[3];
  int ne[3], N;
  int py;
  long long pz;
  double x[DG_MAXN + 1], bw[DG_MAXN + 1];   // GLL nodes and barycentric weights
};
struct NaArgs {
  int R, nd;
  NaBox box[2];
  unsigned char* scratch;
};

__device__ void na_lagrange(const NaBox& B, double t, double* out) {
  const int N = B.N;
  for (int j = 0; j <= N; ++j)
    if (t == B.x[j]) {
      for (int k = 0; k <= N; ++k) out[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int j = 0; j <= N; ++j) den += B.bw[j] / (t - B.x[j]);
  for (int j = 0; j <= N; ++j) out[j] = (B.bw[j] / (t - B.x[j])) / den;
}

// One thread per receiver: containing element (primary box first, lowest
// element id on ties) and its tensor Lagrange weights, written to the table.
__global__ void na_receiver_table(const __grid_constant__ NaArgs A) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.R) return;
  const double* xyz = reinterpret_cast<const double*>(A.scratch + NA_OFF_XYZ) + 3 * r;
  double* w = reinterpret_cast<double*>(A.scratch + NA_OFF_W) + (size_t)r * NA_MAX_NODES;
  long long* off = reinterpret_cast<long long*>(A.scratch + NA_OFF_OFF) + (size_t)r * NA_MAX_NODES;
  int* dom = reinterpret_cast<int*>(A.scratch + NA_OFF_DOM);
  int* nn = reinterpret_cast<int*>(A.scratch + NA_OFF_NN);
  int found = -1;
  for (int d = 0; d < A.nd && found < 0; ++d) {
    bool inside = true;
    for (int k = 0; k < 3; ++k) {
      const double t = 1e-12 * A.box[d].ext[k];
      if (xyz[k] < A.box[d].o[k] - t || xyz[k] > A.box[d].o[k] + A.box[d].ext[k] + t) inside = false;
    }
    if (inside) found = d;
  }
  if (found < 0) {
    atomicExch(reinterpret_cast<int*>(A.scratch + NA_OFF_STATUS), r + 1);
    nn[r] = 0;
    dom[r] = 0;
    return;
  }
  const NaBox& B = A.box[found];
  int e[3];
  double ref[3];
  for (int k = 0; k < 3; ++k) {
    const double u = (xyz[k] - B.o[k]) / B.h[k];
    int ek = (int)ceil(u - 1e-12) - 1;
    ek = max(0, min(ek, B.ne[k] - 1));
    e[k] = ek;
    ref[k] = fmax(-1.0, fmin(1.0, 2.0 * (u - ek) - 1.0));
  }
  double lx[DG_MAXN + 1], ly[DG_MAXN + 1], lz[DG_MAXN + 1];
  na_lagrange(B, ref[0], lx);
  na_lagrange(B, ref[1], ly);
  na_lagrange(B, ref[2], lz);
  const int n1 = B.N + 1;
  int t = 0;
  for (int cc = 0; cc < n1; ++cc)
    for (int bb = 0; bb < n1; ++bb)
      for (int aa = 0; aa < n1; ++aa, ++t) {
        w[t] = lx[aa] * ly[bb] * lz[cc];
        off[t] = (long long)(e[2] * B.N + cc) * B.pz + (long long)(e[1] * B.N + bb) * B.py + (e[0] * B.N + aa);
      }
  dom[r] = found;
  nn[r] = t;
}

}  // namespace

extern "C" int dgsem_sample_noalloc(dgsem_ctx* c, int n_recv, const double* recv_xyz, double* out, size_t out_len,
                                    void* stream) {
  if (!c) return fail(DGSEM_EINVAL, "ctx is NULL");
  if (n_recv < 0 || n_recv > NA_MAX_RECV)
    return fail(DGSEM_EINVAL, "dgsem_sample_noalloc: n_recv = %d outside [0, %d] (its receiver table holds at most %d points)",
                n_recv, NA_MAX_RECV, NA_MAX_RECV);
  if (n_recv == 0) return DGSEM_OK;
  if (!recv_xyz || !out) return fail(DGSEM_EINVAL, "recv_xyz and out are required");
  if (!c->state_valid || !c->X[0]) return fail(DGSEM_ESTATE, "no pressure state: call dgsem_run first");
  if (out_len < (size_t)c->batch * (size_t)n_recv)
    return fail(DGSEM_EINVAL, "out holds %zu doubles, [batch = %d][n_recv = %d] needs %zu", out_len, c->batch, n_recv,
                (size_t)c->batch * (size_t)n_recv);
  if (!is_device_ptr(out)) return fail(DGSEM_EINVAL, "out must be device memory ([batch][n_recv] doubles)");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != c->device) return fail(DGSEM_EINVAL, "context belongs to device %d, current is %d", c->device, dev);
  if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(DGSEM_EINVAL, "device %d beyond the supported %d", dev, NA_MAX_DEVICES);
  // set-up, once per device: the device address of the scratch array (the
  // host-side symbol is only a stand-in and must never reach a kernel)
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_sample_scratch_mu);
    if (!g_sample_scratch_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_sample_scratch);
      if (e != cudaSuccess || !ptr)
        return fail(DGSEM_ECUDA, "cudaGetSymbolAddress(g_sample_scratch): %s", cudaGetErrorString(e));
      g_sample_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
    }
    scratch = g_sample_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the status word must start at zero; the table entries are overwritten
  CUDA_TRY(cudaMemsetAsync(scratch + NA_OFF_STATUS, 0, sizeof(int), s));
  CUDA_TRY(cudaMemcpyAsync(scratch + NA_OFF_XYZ, recv_xyz, (size_t)n_recv * 3 * sizeof(double), cudaMemcpyDefault, s));
  NaArgs a;
  std::memset(&a, 0, sizeof(a));
  a.R = n_recv;
  a.nd = c->nd;
  a.scratch = scratch;
  for (int d = 0; d < c->nd; ++d) {
    const Box& B = c->box[d];
    for (int k = 0; k < 3; ++k) {
      a.box[d].o[k] = B.o[k]; a.box[d].h[k] = B.h[k]; a.box[d].ext[k] = B.ext[k]; a.box[d].ne[k] = B.ne[k];
    }
    a.box[d].N = B.N;
    a.box[d].py = B.py;
    a.box[d].pz = B.pz;
    for (int i = 0; i <= B.N; ++i) { a.box[d].x[i] = B.basis->x[i]; a.box[d].bw[i] = B.basis->bw[i]; }
  }
  na_receiver_table<<<(n_recv + 63) / 64, 64, 0, s>>>(a);
  CUDA_TRY(cudaGetLastError());
  int status = 0;
  CUDA_TRY(cudaMemcpyAsync(&status, scratch + NA_OFF_STATUS, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (status) return fail(DGSEM_EINVAL, "receiver %d is outside the mesh", status - 1);
  // the receiver-sampling kernel of the time loop, reading the table from the scratch array
  cudaError_t e;
  if (c->prec == DGSEM_FP32_MIXED) {
    PmutArgs<float> p;
    std::memset(&p, 0, sizeof(p));
    p.B = c->batch; p.K = 0; p.R = n_recv; p.rstride = NA_MAX_NODES;
    p.rw = reinterpret_cast<const double*>(scratch + NA_OFF_W);
    p.roff = reinterpret_cast<const long long*>(scratch + NA_OFF_OFF);
    p.rdom = reinterpret_cast<const int*>(scratch + NA_OFF_DOM);
    p.rnn = reinterpret_cast<const int*>(scratch + NA_OFF_NN);
    p.pc0 = static_cast<const float*>(c->X[0]); p.pc1 = c->nd > 1 ? static_cast<const float*>(c->X[1]) : nullptr;
    p.bs0 = c->box[0].bstride; p.bs1 = c->nd > 1 ? c->box[1].bstride : 0;
    p.traces = out; p.tbs = n_recv; p.trs = 1; p.n = 0; p.step = nullptr;
    e = launch_pmut_recv<float>(p, s);
  } else {
    PmutArgs<double> p;
    std::memset(&p, 0, sizeof(p));
    p.B = c->batch; p.K = 0; p.R = n_recv; p.rstride = NA_MAX_NODES;
    p.rw = reinterpret_cast<const double*>(scratch + NA_OFF_W);
    p.roff = reinterpret_cast<const long long*>(scratch + NA_OFF_OFF);
    p.rdom = reinterpret_cast<const int*>(scratch + NA_OFF_DOM);
    p.rnn = reinterpret_cast<const int*>(scratch + NA_OFF_NN);
    p.pc0 = static_cast<const double*>(c->X[0]); p.pc1 = c->nd > 1 ? static_cast<const double*>(c->X[1]) : nullptr;
    p.bs0 = c->box[0].bstride; p.bs1 = c->nd > 1 ? c->box[1].bstride : 0;
    p.traces = out; p.tbs = n_recv; p.trs = 1; p.n = 0; p.step = nullptr;
    e = launch_pmut_recv<double>(p, s);
  }
  if (e != cudaSuccess) return fail(DGSEM_ECUDA, "receiver sampling launch: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaStreamSynchronize(s));
  return DGSEM_OK;
}
