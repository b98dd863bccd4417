// Host setup and C ABI of the DG-SEM step on general hexahedral meshes
// (include/dghex.h).
//
// Setup (untimed): topological C0 numbering of the GLL nodes of each domain
// (shared vertices, edges and faces matched by vertex ids, any element
// orientation), geometric factors and lumped mass on the GPU, Algorithm 3 on
// the GPU, the slot layout of the element-local residuals, PMUT face weights,
// receivers and the time step.
// Step: PMUT modal step (the box path's kernel), element stiffness of each
// domain, interface terms, residual gather + leapfrog update, tail (forcing
// slots, receivers, step counter) -- Algorithm 1 in two-vector leapfrog form
// with the state (p^n, v^{n-1/2}).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/dghex.h"
#include "hex_geom.h"
#include "internal.h"
#include "tables.h"

namespace {

int hfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return dg_fail_msg(code, buf);
}

#define HCUDA(expr)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return hfail(e_ == cudaErrorMemoryAllocation ? DGSEM_ENOMEM : DGSEM_ECUDA,         \
                   "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

template <typename P>
int dmalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return DGSEM_OK;
  HCUDA(cudaMalloc(reinterpret_cast<void**>(p), bytes));
  return DGSEM_OK;
}

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree(const_cast<void*>(reinterpret_cast<const void*>(p)));
  p = nullptr;
}

template <typename V>
int upload(V** d, const std::vector<V>& h) {
  int rc = dmalloc(d, h.size() * sizeof(V));
  if (rc) return rc;
  if (!h.empty()) HCUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
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

struct HexDom {
  int N = 0, n = 0, nl = 0, ne = 0, nv = 0;
  double c = 0.0, rho = 0.0;
  std::vector<double> vert;
  std::vector<int> elem;
  std::vector<int> conn;          // [ne][nl] global node ids
  long long node0 = 0, nnode = 0;
  long long vslot0 = 0;           // first volume slot
  dgtab::Basis1D* basis = nullptr;
  double* d_vert = nullptr;
  int* d_elem = nullptr;
  int* d_conn = nullptr;
  double* d_G64 = nullptr;
  float* d_G32 = nullptr;
  // perfectly matched layer: thickness per bounding-box side, layer elements,
  // their J^-1 and w |J| at the GLL nodes, first layer slot
  double pml_th[6] = {0, 0, 0, 0, 0, 0};
  std::vector<int> pml_elem;
  int* d_pml_elem = nullptr;
  double* d_pml_geo64 = nullptr; float* d_pml_geo32 = nullptr;
  long long pslot0 = 0;
  void* Phi = nullptr;                 // run state [npml][3][nl][Bp]
};

// corner list position of the corner with bits (i, j, k)
inline int corner(int i, int j, int k) { return i + 2 * j + 4 * k; }

// C0 numbering of one domain's GLL nodes: vertices, edges (keyed by their two
// vertex ids, counted from the smaller), faces (keyed by the smallest vertex
// and its two face neighbours, counted from the smallest towards the smaller
// neighbour first) and element interiors.  Ids are assigned in order of first
// appearance of the entity over the elements.
int number_nodes(HexDom& D, long long node0, std::map<std::array<int, 4>, int>& face_count) {
  const int N = D.N, n = D.n, nl = D.nl;
  D.conn.assign((size_t)D.ne * nl, -1);
  std::vector<long long> vnode(D.nv, -1);
  std::unordered_map<unsigned long long, long long> edge_base;
  std::map<std::array<int, 3>, long long> face_base;
  long long next = 0;
  const long long nv = D.nv;
  for (int e = 0; e < D.ne; ++e) {
    const int* V = &D.elem[(size_t)e * 8];
    for (int f = 0; f < 6; ++f) {
      const int ax = f >> 1, side = f & 1;
      std::array<int, 4> key;
      int k = 0;
      for (int c = 0; c < 8; ++c)
        if (((c >> ax) & 1) == side) key[k++] = V[c];
      std::sort(key.begin(), key.end());
      face_count[key] += 1;
    }
    long long ibase = -1;
    for (int i = 0; i < nl; ++i) {
      const int l[3] = {i % n, (i / n) % n, i / (n * n)};
      bool ext[3];
      int next_ax = 0;
      for (int d = 0; d < 3; ++d) {
        ext[d] = l[d] == 0 || l[d] == N;
        next_ax += ext[d];
      }
      long long id;
      if (next_ax == 3) {
        const int v = V[corner(l[0] == N, l[1] == N, l[2] == N)];
        if (vnode[v] < 0) vnode[v] = next++;
        id = vnode[v];
      } else if (next_ax == 2) {
        const int fa = !ext[0] ? 0 : (!ext[1] ? 1 : 2);
        int bits[3] = {l[0] == N, l[1] == N, l[2] == N};
        bits[fa] = 0;
        const int vA = V[corner(bits[0], bits[1], bits[2])];
        bits[fa] = 1;
        const int vB = V[corner(bits[0], bits[1], bits[2])];
        const unsigned long long key = (unsigned long long)std::min(vA, vB) * (unsigned long long)nv + std::max(vA, vB);
        auto it = edge_base.find(key);
        long long base;
        if (it == edge_base.end()) {
          base = next;
          next += N - 1;
          edge_base.emplace(key, base);
        } else {
          base = it->second;
        }
        const int t = l[fa];
        id = base + (vA < vB ? t - 1 : N - 1 - t);
      } else if (next_ax == 1) {
        const int xa = ext[0] ? 0 : (ext[1] ? 1 : 2);
        const int f1 = xa == 0 ? 1 : 0, f2 = xa == 2 ? 1 : 2;
        const int s = l[xa] == N;
        auto C = [&](int i1, int i2) {
          int bits[3];
          bits[xa] = s;
          bits[f1] = i1;
          bits[f2] = i2;
          return V[corner(bits[0], bits[1], bits[2])];
        };
        int oi = 0, oj = 0;
        for (int i1 = 0; i1 < 2; ++i1)
          for (int i2 = 0; i2 < 2; ++i2)
            if (C(i1, i2) < C(oi, oj)) {
              oi = i1;
              oj = i2;
            }
        const int n1 = C(1 - oi, oj), n2 = C(oi, 1 - oj);
        const int u = oi == 0 ? l[f1] : N - l[f1];
        const int w = oj == 0 ? l[f2] : N - l[f2];
        int first, second;
        std::array<int, 3> key;
        if (n1 < n2) {
          first = u; second = w; key = {C(oi, oj), n1, n2};
        } else {
          first = w; second = u; key = {C(oi, oj), n2, n1};
        }
        auto it = face_base.find(key);
        long long base;
        if (it == face_base.end()) {
          base = next;
          next += (long long)(N - 1) * (N - 1);
          face_base.emplace(key, base);
        } else {
          base = it->second;
        }
        id = base + (first - 1) + (long long)(N - 1) * (second - 1);
      } else {
        if (ibase < 0) {
          ibase = next;
          next += (long long)(N - 1) * (N - 1) * (N - 1);
        }
        id = ibase + (l[0] - 1) + (long long)(N - 1) * ((l[1] - 1) + (long long)(N - 1) * (l[2] - 1));
      }
      D.conn[(size_t)e * nl + i] = (int)(node0 + id);
    }
  }
  D.node0 = node0;
  D.nnode = next;
  return DGSEM_OK;
}

void elem_verts(const HexDom& D, int e, double* V) {
  for (int c = 0; c < 8; ++c)
    for (int k = 0; k < 3; ++k) V[3 * c + k] = D.vert[3 * (size_t)D.elem[(size_t)e * 8 + c] + k];
}

}  // namespace

struct dghex_ctx {
  int device = 0;
  int nd = 0;
  HexDom dom[2];
  long long ndof = 0, nvol = 0;
  std::vector<double> xyz;
  double dt = 0.0;
  double dt_cfl = 0.0;                      // dt before the absorbing-face limit
  bool dt_fixed = false;                    // dt given by the caller
  std::vector<std::map<std::array<int, 4>, int>> fcount;   // element faces per domain (boundary test)
  std::vector<double> Mh;                   // lumped mass (host copy)
  // absorbing faces per domain, and C_jj / M_jj on the device (NULL: none)
  std::vector<int> abs_faces[2];
  double* d_damp64 = nullptr; float* d_damp32 = nullptr;   // C_jj/M_jj + alpha_j
  // perfectly matched layers: design reflection, profiles zeta_d per node and
  // the node coefficients beta, gamma (alpha is in the damping array)
  bool has_pml = false;
  double pml_R = 1e-4;
  double *d_zeta64 = nullptr, *d_beta64 = nullptr, *d_gamma64 = nullptr;
  float *d_zeta32 = nullptr, *d_beta32 = nullptr, *d_gamma32 = nullptr;
  long long npslot = 0;                     // layer slots (after the forcing slots)
  std::vector<double> pml_alpha;            // alpha_j per node (host)
  void* Psi = nullptr;                      // run state [ndof][Bp]
  // TX -> RX switch of the PMUT array (off: rx_switch < 0)
  long long rx_switch = -1;
  double* d_rx_gain = nullptr;
  long long* d_step_base = nullptr;        // steps done before the current run
  long long steps_done = 0;                 // steps since rest or the last set state
  double* d_volt = nullptr; size_t volt_cap = 0; long long volt_n = 0;
  // interface (Algorithm 3)
  int q = 0, nff = 0, ncf = 0;
  std::vector<int> ff, cf, match;
  std::vector<double> refm;
  int ng = 0, max_pts = 0;
  long long islot0 = 0, nislot = 0;
  std::vector<int> g_fe, g_ce, g_pt, pt_idx, g_face;
  bool onface = false;                      // every group's Gauss nodes lie on one face per side
  bool force_general_iface = false;         // use the general interface kernel even when onface
  int vol_variant[2][2] = {};               // element-stiffness launch variant [FP64, FP32][domain]
  int* d_g_face = nullptr;
  void* d_ftab[2] = {nullptr, nullptr};     // face-kernel per-point tables [FP64, FP32] (built on first use)
  void* d_gtab[2] = {nullptr, nullptr};     // general-kernel per-point tables [FP64, FP32] (built on first use)
  std::vector<long long> g_slot;
  int *d_g_fe = nullptr, *d_g_ce = nullptr, *d_g_pt = nullptr, *d_pt_idx = nullptr;
  long long* d_g_slot = nullptr;
  double* d_pdat = nullptr;
  // Gamma_PMUT
  std::vector<long long> pn_id;
  std::vector<double> pn_xyz, pn_w;
  int K = 0, M = 0, nnz = 0;
  long long fslot0 = 0;
  std::vector<long long> ent_node;
  std::vector<int> pmut_faces;
  int* d_fp_ptr = nullptr; long long* d_fp_off = nullptr; double* d_Bm = nullptr; int* d_ent_k = nullptr;
  double* d_modal = nullptr;
  double kappa = 0.0;
  // slots and their per-node lists
  long long nslot = 0;
  int* d_node_ptr = nullptr; int* d_node_slot = nullptr;
  double* d_Mloc = nullptr; double* d_M = nullptr; double* d_Minv64 = nullptr; float* d_Minv32 = nullptr;
  // run state: fields batch-innermost, row length Bp (the batch padded to a
  // multiple of the 32-byte vector width when it is at least that wide)
  int prec = -1, batch = 0, Bp = 0;
  // X = p^n, Y = p^{n+1}, V = v^{n+1/2} (two-vector form of Algorithm 1;
  // X and Y swap every step)
  void* X = nullptr; void* Y = nullptr; void* V = nullptr; void* S = nullptr;
  long long* d_fp_offB = nullptr;          // footprint node offsets j * Bp for the PMUT kernel
  double* q_state = nullptr;
  bool state_valid = false;
  int* d_step = nullptr; unsigned* d_done = nullptr;
  int* d_nf = nullptr;                      // non-finite flag of the divergence check
  std::vector<double> init_p, init_v;
  bool has_init = false;
  // receivers and scratch for host-pointer runs
  double* d_rw = nullptr; long long* d_roff = nullptr; int* d_rnn = nullptr;
  size_t recv_cap = 0; int rstride = 0;
  std::vector<double> recv_xyz;            // positions the receiver tables were built for
  double* d_drive = nullptr; size_t drive_cap = 0;
  double* d_traces = nullptr; size_t traces_cap = 0;
  // instrumentation
  bool profiling = false;
  long long launches[DGHEX_K_COUNT] = {};
  double kernel_ms[DGHEX_K_COUNT] = {};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;
};

namespace {

struct HexTimer {
  dghex_ctx* c; cudaStream_t s; int kind; int idx = -1;
  HexTimer(dghex_ctx* c_, cudaStream_t s_, int k) : c(c_), s(s_), kind(k) {
    c->launches[kind] += 1;
    if (!c->profiling) return;
    idx = (int)c->ev_used.size() * 2;
    while ((int)c->ev_pool.size() < idx + 2) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) { idx = -1; return; }
      c->ev_pool.push_back(ev);
    }
    cudaEventRecord(c->ev_pool[idx], s);
  }
  ~HexTimer() {
    if (idx < 0) return;
    cudaEventRecord(c->ev_pool[idx + 1], s);
    c->ev_used.emplace_back(kind, idx);
  }
};

void collect_timings(dghex_ctx* c) {
  for (auto& u : c->ev_used) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[u.second], c->ev_pool[u.second + 1]) == cudaSuccess)
      c->kernel_ms[u.first] += ms;
  }
  c->ev_used.clear();
}

void free_run_state(dghex_ctx* c) {
  dfree(c->X); dfree(c->Y); dfree(c->V); dfree(c->S); dfree(c->q_state); dfree(c->d_fp_offB);
  dfree(c->Psi);
  for (int d = 0; d < 2; ++d) dfree(c->dom[d].Phi);
  c->prec = -1;
  c->batch = 0;
  c->Bp = 0;
  c->state_valid = false;
}

int ensure_run_state(dghex_ctx* c, int prec, int batch) {
  if (c->prec == prec && c->batch == batch && c->X) return DGSEM_OK;
  free_run_state(c);
  const size_t es = prec == DGSEM_FP32_MIXED ? sizeof(float) : sizeof(double);
  const int vw = (int)(32 / es);
  const int Bp = batch < vw ? batch : (batch + vw - 1) / vw * vw;
  int rc;
  if ((rc = dmalloc(&c->X, es * Bp * c->ndof)) || (rc = dmalloc(&c->Y, es * Bp * c->ndof)) ||
      (rc = dmalloc(&c->V, es * Bp * c->ndof)) ||
      (rc = dmalloc(&c->S, es * Bp * c->nslot)))
    return rc;
  if (c->has_pml) {
    if ((rc = dmalloc(&c->Psi, es * Bp * c->ndof))) return rc;
    for (int d = 0; d < c->nd; ++d)
      if ((rc = dmalloc(&c->dom[d].Phi, es * Bp * 3 * c->dom[d].nl * c->dom[d].pml_elem.size()))) return rc;
  }
  if (c->K > 0) {
    if ((rc = dmalloc(&c->q_state, sizeof(double) * 3 * (size_t)batch * c->K * c->M))) return rc;
    std::vector<long long> off(c->ent_node);
    for (auto& o : off) o *= Bp;
    if ((rc = upload(&c->d_fp_offB, off))) return rc;
  }
  c->prec = prec;
  c->batch = batch;
  c->Bp = Bp;
  return DGSEM_OK;
}

// Slot layout: volume slots of domain 0 then 1 (element-major), the interface
// groups' blocks, then one forcing slot per PMUT footprint entry; each node
// lists its slots in ascending order.
int build_slots(dghex_ctx* c) {
  c->islot0 = c->nvol;
  c->fslot0 = c->islot0 + c->nislot;
  long long ps = c->fslot0 + c->nnz;
  for (int d = 0; d < c->nd; ++d) {
    c->dom[d].pslot0 = ps;
    ps += (long long)c->dom[d].pml_elem.size() * c->dom[d].nl;
  }
  c->npslot = ps - c->fslot0 - c->nnz;
  c->nslot = ps;
  if (c->nslot >= (1LL << 31)) return hfail(DGSEM_EINVAL, "mesh too large: %lld residual slots", c->nslot);
  std::vector<int> node_of((size_t)c->nslot);
  for (int d = 0; d < c->nd; ++d) {
    const HexDom& D = c->dom[d];
    for (size_t k = 0; k < D.conn.size(); ++k) node_of[(size_t)D.vslot0 + k] = D.conn[k];
  }
  if (c->nd == 2) {
    const HexDom &Dp = c->dom[0], &Dm = c->dom[1];
    for (int g = 0; g < c->ng; ++g) {
      const long long s0 = c->g_slot[g];
      for (int i = 0; i < Dp.nl; ++i) node_of[s0 + i] = Dp.conn[(size_t)c->g_fe[g] * Dp.nl + i];
      for (int i = 0; i < Dm.nl; ++i) node_of[s0 + Dp.nl + i] = Dm.conn[(size_t)c->g_ce[g] * Dm.nl + i];
    }
  }
  for (int e = 0; e < c->nnz; ++e) node_of[(size_t)c->fslot0 + e] = (int)c->ent_node[e];
  for (int d = 0; d < c->nd; ++d) {
    const HexDom& D = c->dom[d];
    for (size_t k = 0; k < D.pml_elem.size(); ++k)
      for (int i = 0; i < D.nl; ++i) node_of[(size_t)D.pslot0 + k * D.nl + i] = D.conn[(size_t)D.pml_elem[k] * D.nl + i];
  }
  std::vector<int> ptr((size_t)c->ndof + 1, 0), slot((size_t)c->nslot);
  for (long long s = 0; s < c->nslot; ++s) ptr[node_of[s] + 1] += 1;
  for (long long j = 0; j < c->ndof; ++j) ptr[j + 1] += ptr[j];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (long long s = 0; s < c->nslot; ++s) slot[fill[node_of[s]]++] = (int)s;
  dfree(c->d_node_ptr);
  dfree(c->d_node_slot);
  int rc;
  if ((rc = upload(&c->d_node_ptr, ptr)) || (rc = upload(&c->d_node_slot, slot))) return rc;
  free_run_state(c);
  return DGSEM_OK;
}

int setup_interface(dghex_ctx* c, const dghex_mesh_desc* d) {
  HexDom &Dp = c->dom[0], &Dm = c->dom[1];
  c->nff = d->n_fine_faces;
  c->ncf = d->n_coarse_faces;
  c->ff.assign(d->fine_faces, d->fine_faces + 2 * (size_t)c->nff);
  c->cf.assign(d->coarse_faces, d->coarse_faces + 2 * (size_t)c->ncf);
  const int q = d->iface_quad_pts > 0 ? d->iface_quad_pts : std::max(Dp.N, Dm.N) + 1;
  if (q > hex::MAXQ) return hfail(DGSEM_EINVAL, "iface_quad_pts %d > %d", q, hex::MAXQ);
  c->q = q;
  std::vector<double> gx, gw;
  dgtab::gauss(q, gx, gw);
  int* d_ff = nullptr; int* d_cf = nullptr;
  double *d_fdat = nullptr, *d_cdat = nullptr, *d_refm = nullptr;
  int* d_match = nullptr;
  const long long npt = (long long)c->nff * q * q;
  int rc;
  auto cleanup = [&]() { dfree(d_ff); dfree(d_cf); dfree(d_fdat); dfree(d_cdat); dfree(d_refm); dfree(d_match); };
  if ((rc = upload(&d_ff, c->ff)) || (rc = upload(&d_cf, c->cf)) || (rc = dmalloc(&d_fdat, 8 * sizeof(double) * c->nff)) ||
      (rc = dmalloc(&d_cdat, 8 * sizeof(double) * c->ncf)) || (rc = dmalloc(&d_refm, 3 * sizeof(double) * npt)) ||
      (rc = dmalloc(&d_match, sizeof(int) * npt)) || (rc = dmalloc(&c->d_pdat, hex::PDAT * sizeof(double) * npt))) {
    cleanup();
    return rc;
  }
  for (int side = 0; side < 2; ++side) {
    HexDom& D = side == 0 ? Dp : Dm;
    hex::FaceArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vert = D.d_vert; a.elem = D.d_elem;
    a.faces = side == 0 ? d_ff : d_cf;
    a.nf = side == 0 ? c->nff : c->ncf;
    a.n = D.n;
    for (int i = 0; i < D.n; ++i) { a.xi[i] = D.basis->x[i]; a.w[i] = D.basis->w[i]; }
    a.Mloc = c->d_Mloc + D.vslot0;
    a.out = side == 0 ? d_fdat : d_cdat;
    cudaError_t e = hex::launch_faces(a, 0);
    if (e != cudaSuccess) { cleanup(); return hfail(DGSEM_ECUDA, "face kernel: %s", cudaGetErrorString(e)); }
  }
  hex::MatchArgs m;
  std::memset(&m, 0, sizeof(m));
  m.vert_p = Dp.d_vert; m.elem_p = Dp.d_elem; m.ff = d_ff; m.fdat = d_fdat;
  m.vert_m = Dm.d_vert; m.elem_m = Dm.d_elem; m.cf = d_cf; m.cdat = d_cdat;
  m.nff = c->nff; m.ncf = c->ncf; m.q = q;
  for (int i = 0; i < q; ++i) { m.g[i] = gx[i]; m.gw[i] = gw[i]; }
  m.tol = d->normal_tol > 0.0 ? d->normal_tol : 0.5;
  m.eps = 1e-12;
  m.match = d_match; m.refm = d_refm;
  const double cbar = 2.0 * Dp.c * Dm.c / (Dp.c + Dm.c);
  const int Nmax = std::max(Dp.N, Dm.N);
  m.alpha_cbar2_n2 = d->penalty_alpha * cbar * cbar * Nmax * Nmax;
  m.pdat = c->d_pdat;
  cudaError_t e = hex::launch_match(m, 0);
  if (e == cudaSuccess) e = hex::launch_ipoints(m, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cleanup(); return hfail(DGSEM_ECUDA, "interface matching: %s", cudaGetErrorString(e)); }
  c->match.resize(npt);
  c->refm.resize(3 * npt);
  e = cudaMemcpy(c->match.data(), d_match, sizeof(int) * npt, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(c->refm.data(), d_refm, 3 * sizeof(double) * npt, cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) return hfail(DGSEM_ECUDA, "interface matching: %s", cudaGetErrorString(e));
  for (long long t = 0; t < npt; ++t)
    if (c->match[t] < 0)
      return hfail(DGSEM_ENOMATCH, "fine face %lld, Gauss node %lld has no coarse neighbour (Algorithm 3)",
                   t / (q * q), t % (q * q));
  // groups: per fine face, its nodes split by coarse element (first appearance)
  c->g_fe.clear(); c->g_ce.clear(); c->g_pt.assign(1, 0); c->pt_idx.clear(); c->g_slot.clear();
  c->g_face.clear();
  c->onface = true;
  long long slot = c->nvol;
  c->max_pts = 0;
  for (int f = 0; f < c->nff; ++f) {
    std::vector<int> ces;
    for (int j = 0; j < q * q; ++j) {
      const int ce = c->cf[2 * c->match[(size_t)f * q * q + j]];
      if (std::find(ces.begin(), ces.end(), ce) == ces.end()) ces.push_back(ce);
    }
    for (int ce : ces) {
      int cnt = 0, cface = -1;
      for (int j = 0; j < q * q; ++j) {
        const size_t t = (size_t)f * q * q + j;
        if (c->cf[2 * c->match[t]] != ce) continue;
        c->pt_idx.push_back((int)t);
        ++cnt;
        // on the matched coarse face: one face for the whole group, and the
        // Newton reference position on it to rounding
        const int lf = c->cf[2 * c->match[t] + 1];
        if (cface < 0) cface = lf;
        const double want = (lf & 1) ? 1.0 : -1.0;
        if (lf != cface || std::fabs(c->refm[3 * t + (lf >> 1)] - want) > 1e-12) c->onface = false;
      }
      c->g_fe.push_back(c->ff[2 * f]);
      c->g_ce.push_back(ce);
      c->g_face.push_back(c->ff[2 * f + 1]);
      c->g_face.push_back(cface);
      c->g_pt.push_back((int)c->pt_idx.size());
      c->g_slot.push_back(slot);
      slot += Dp.nl + Dm.nl;
      c->max_pts = std::max(c->max_pts, cnt);
    }
  }
  c->ng = (int)c->g_fe.size();
  c->nislot = slot - c->nvol;
  if ((rc = upload(&c->d_g_fe, c->g_fe)) || (rc = upload(&c->d_g_ce, c->g_ce)) || (rc = upload(&c->d_g_pt, c->g_pt)) ||
      (rc = upload(&c->d_pt_idx, c->pt_idx)) || (rc = upload(&c->d_g_slot, c->g_slot)) ||
      (rc = upload(&c->d_g_face, c->g_face)))
    return rc;
  return DGSEM_OK;
}

// Unique nodes of the PMUT faces with W_j = sum_F w_a w_b |J_F| (host, FP64).
void setup_pmut_nodes(dghex_ctx* c, const std::vector<int>& faces) {
  const HexDom& D = c->dom[0];
  std::map<long long, double> W;
  std::map<long long, std::array<double, 3>> X;
  for (size_t k = 0; k < faces.size() / 2; ++k) {
    const int e = faces[2 * k], f = faces[2 * k + 1];
    double V[24];
    elem_verts(D, e, V);
    const int ax = f >> 1, fixed = (f & 1) ? D.N : 0;
    const int t0 = ax == 0 ? 1 : 0, t1 = ax == 2 ? 1 : 2;
    for (int i = 0; i < D.nl; ++i) {
      const int l[3] = {i % D.n, (i / D.n) % D.n, i / (D.n * D.n)};
      if (l[ax] != fixed) continue;
      const double r[3] = {D.basis->x[l[0]], D.basis->x[l[1]], D.basis->x[l[2]]};
      double x[3], J[3][3], nrm[3];
      hex::tri_map(V, r, x, J);
      const double dS = hex::face_normal(f, J, nrm);
      const long long id = D.conn[(size_t)e * D.nl + i];
      W[id] += D.basis->w[l[t0]] * D.basis->w[l[t1]] * dS;
      X[id] = {x[0], x[1], x[2]};
    }
  }
  c->pn_id.clear(); c->pn_xyz.clear(); c->pn_w.clear();
  for (auto& kv : W) {
    c->pn_id.push_back(kv.first);
    c->pn_w.push_back(kv.second);
    const auto& x = X[kv.first];
    c->pn_xyz.insert(c->pn_xyz.end(), x.begin(), x.end());
  }
}

// Receivers: lowest-id containing element (primary first), tensor Lagrange
// weights at the Newton reference position.
int setup_receivers(dghex_ctx* c, int R, const double* xyz) {
  if (R == 0) return DGSEM_OK;
  if (c->recv_xyz.size() == 3 * (size_t)R && std::equal(c->recv_xyz.begin(), c->recv_xyz.end(), xyz))
    return DGSEM_OK;
  c->recv_xyz.clear();
  int maxn = 0;
  for (int d = 0; d < c->nd; ++d) maxn = std::max(maxn, c->dom[d].nl);
  std::vector<double> w((size_t)R * maxn, 0.0);
  std::vector<long long> off((size_t)R * maxn, 0);
  std::vector<int> nn(R, 0);
  for (int r = 0; r < R; ++r) {
    const double* x = xyz + 3 * (size_t)r;
    bool done = false;
    for (int d = 0; d < c->nd && !done; ++d) {
      const HexDom& D = c->dom[d];
      for (int e = 0; e < D.ne && !done; ++e) {
        double V[24];
        elem_verts(D, e, V);
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int k = 0; k < 8; ++k)
          for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], V[3 * k + a]);
            hi[a] = std::max(hi[a], V[3 * k + a]);
          }
        const double pad = 1e-9 * std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        bool out = false;
        for (int a = 0; a < 3; ++a) out = out || x[a] < lo[a] - pad || x[a] > hi[a] + pad;
        if (out) continue;
        double ref[3];
        if (!hex::newton_ref(V, x, ref) || !hex::inside_ref(ref)) continue;
        double l[3][hex::MAXN1], dl[hex::MAXN1];
        for (int a = 0; a < 3; ++a) hex::lagrange(D.n, D.basis->x.data(), std::min(1.0, std::max(-1.0, ref[a])), l[a], dl);
        for (int i = 0; i < D.nl; ++i) {
          w[(size_t)r * maxn + i] = l[0][i % D.n] * l[1][(i / D.n) % D.n] * l[2][i / (D.n * D.n)];
          off[(size_t)r * maxn + i] = D.conn[(size_t)e * D.nl + i];
        }
        nn[r] = D.nl;
        done = true;
      }
    }
    if (!done) return hfail(DGSEM_EINVAL, "receiver %d (%g, %g, %g) is outside the mesh", r, x[0], x[1], x[2]);
  }
  if ((size_t)R > c->recv_cap || maxn != c->rstride) {
    dfree(c->d_rw); dfree(c->d_roff); dfree(c->d_rnn);
    int rc;
    if ((rc = dmalloc(&c->d_rw, sizeof(double) * R * maxn)) || (rc = dmalloc(&c->d_roff, sizeof(long long) * R * maxn)) ||
        (rc = dmalloc(&c->d_rnn, sizeof(int) * R)))
      return rc;
    c->recv_cap = R;
  }
  c->rstride = maxn;
  HCUDA(cudaMemcpy(c->d_rw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  HCUDA(cudaMemcpy(c->d_roff, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
  HCUDA(cudaMemcpy(c->d_rnn, nn.data(), nn.size() * sizeof(int), cudaMemcpyHostToDevice));
  c->recv_xyz.assign(xyz, xyz + 3 * (size_t)R);
  return DGSEM_OK;
}

// element stiffness of domain d applied to the pressure field p
template <typename T>
hex::HexVolArgs<T> vol_args(const dghex_ctx* c, int d, const void* pfield) {
  const HexDom& D = c->dom[d];
  hex::HexVolArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.p = static_cast<const T*>(pfield); a.S = static_cast<T*>(c->S); a.Bp = c->Bp;
  a.conn = D.d_conn;
  a.G = std::is_same<T, float>::value ? reinterpret_cast<const T*>(D.d_G32) : reinterpret_cast<const T*>(D.d_G64);
  a.slot_base = D.vslot0;
  a.ne = D.ne;
  const int n = D.n, h = n / 2;
  for (int t = 0; t < 2; ++t) {
    auto C = [&](int i, int j) { return t == 0 ? D.basis->D[i * n + j] : D.basis->D[j * n + i]; };
    for (int r = 0; r < h; ++r) {
      for (int m = 0; m < h; ++m) {
        a.ea[t][r][m] = T(0.5 * (C(r, m) - C(r, n - 1 - m)));
        a.eb[t][r][m] = T(0.5 * (C(r, m) + C(r, n - 1 - m)));
      }
      if (n % 2 == 1) a.eb[t][r][h] = T(C(r, h));
    }
    if (n % 2 == 1)
      for (int m = 0; m < h; ++m) a.em[t][m] = T(C(h, m));
  }
  return a;
}

template <typename T>
int vol_variant_of(const dghex_ctx* c, int d) { return c->vol_variant[std::is_same<T, float>::value ? 1 : 0][d]; }

// element stiffness and interface terms of the pressure field p
template <typename T>
int launch_residual(dghex_ctx* c, cudaStream_t s, const void* pfield) {
  const T* p = static_cast<const T*>(pfield);
  T* S = static_cast<T*>(c->S);
  for (int d = 0; d < c->nd; ++d) {
    const hex::HexVolArgs<T> a = vol_args<T>(c, d, pfield);
    HexTimer t(c, s, DGHEX_K_VOL);
    HCUDA(hex::launch_hex_vol<T>(a, c->dom[d].n, vol_variant_of<T>(c, d), s));
  }
  if (c->nd == 2 && c->ng > 0) {
    const HexDom &Dp = c->dom[0], &Dm = c->dom[1];
    hex::HexIfaceArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.p = p; a.S = S; a.Bp = c->Bp;
    a.conn_p = Dp.d_conn; a.conn_m = Dm.d_conn;
    a.g_fe = c->d_g_fe; a.g_ce = c->d_g_ce; a.g_pt = c->d_g_pt; a.pt_idx = c->d_pt_idx; a.g_slot = c->d_g_slot;
    a.g_face = c->d_g_face;
    a.onface = c->onface && !c->force_general_iface ? 1 : 0;
    for (int i = 0; i < Dp.n; ++i)
      for (int j = 0; j < Dp.n; ++j) a.Dp[i][j] = T(Dp.basis->D[i * Dp.n + j]);
    for (int i = 0; i < Dm.n; ++i)
      for (int j = 0; j < Dm.n; ++j) a.Dm[i][j] = T(Dm.basis->D[i * Dm.n + j]);
    a.pdat = c->d_pdat;
    for (int i = 0; i < Dp.n; ++i) a.xip[i] = Dp.basis->x[i];
    for (int i = 0; i < Dm.n; ++i) a.xim[i] = Dm.basis->x[i];
    a.np = Dp.n; a.nm = Dm.n;
    a.c2p = Dp.c * Dp.c; a.c2m = Dm.c * Dm.c;
    a.ng = c->ng; a.max_pts = c->max_pts;
    if (a.onface) {
      void*& tab = c->d_ftab[std::is_same<T, float>::value ? 1 : 0];
      if (!tab) {
        int rc = dmalloc(&tab, sizeof(T) * (size_t)hex::kFaceTab * (size_t)c->g_pt[c->ng]);
        if (rc) return rc;
        HCUDA(hex::launch_hex_iface_table<T>(a, static_cast<T*>(tab), s));
      }
      a.ftab = static_cast<const T*>(tab);
    } else {
      void*& tab = c->d_gtab[std::is_same<T, float>::value ? 1 : 0];
      if (!tab) {
        int rc = dmalloc(&tab, sizeof(T) * (size_t)hex::kGenTab * (size_t)c->g_pt[c->ng]);
        if (rc) return rc;
        HCUDA(hex::launch_hex_iface_gtable<T>(a, static_cast<T*>(tab), s));
      }
      a.gtab = static_cast<const T*>(tab);
    }
    HexTimer t(c, s, DGHEX_K_IFACE);
    HCUDA(hex::launch_hex_iface<T>(a, s));
  }
  return DGSEM_OK;
}

// pml: 0 no layer terms, 1 set-state start (psi stays 0), 2 time step
template <typename T>
int launch_update(dghex_ctx* c, cudaStream_t s, double cv, double cp, const void* p_in, void* p_out, int pml = 0,
                  void* v = nullptr) {
  hex::HexUpdateArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.p_in = static_cast<const T*>(p_in); a.p_out = static_cast<T*>(p_out);
  a.v = static_cast<T*>(v ? v : c->V); a.S = static_cast<const T*>(c->S);
  a.Bp = c->Bp;
  a.node_ptr = c->d_node_ptr; a.node_slot = c->d_node_slot;
  a.Minv = std::is_same<T, float>::value ? reinterpret_cast<const T*>(c->d_Minv32) : reinterpret_cast<const T*>(c->d_Minv64);
  a.damp = std::is_same<T, float>::value ? reinterpret_cast<const T*>(c->d_damp32) : reinterpret_cast<const T*>(c->d_damp64);
  if (pml && c->has_pml) {
    const bool f = std::is_same<T, float>::value;
    a.beta = f ? reinterpret_cast<const T*>(c->d_beta32) : reinterpret_cast<const T*>(c->d_beta64);
    a.gamma = f ? reinterpret_cast<const T*>(c->d_gamma32) : reinterpret_cast<const T*>(c->d_gamma64);
    a.psi = static_cast<T*>(c->Psi);
    a.hpsi = pml == 2 ? T(0.5 * c->dt) : T(0);
    a.dpsi = pml == 2 ? T(c->dt) : T(0);
  }
  a.ndof = c->ndof; a.cv = T(cv); a.cp = T(cp);
  HexTimer t(c, s, DGHEX_K_UPDATE);
  HCUDA(hex::launch_hex_update<T>(a, s));
  return DGSEM_OK;
}

// PMUT forcing rows kappa sum_m q''_km B_jm (R = 0) or receivers of Y and the
// step counter (forcing = false)
template <typename T>
int launch_tail(dghex_ctx* c, cudaStream_t s, bool forcing, int R, double* traces, long long tbs, long long trs) {
  hex::HexTailArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.M = c->M; a.K = c->K; a.B = c->batch; a.Bp = c->Bp;
  a.S = static_cast<T*>(c->S); a.fslot = c->fslot0;
  if (forcing) {
    a.nnz = c->nnz;
    a.ent_k = c->d_ent_k; a.Bm = c->d_Bm;
    a.qdd = c->q_state + 2 * (long long)c->batch * c->K * c->M;
    a.kappa = c->kappa;
    a.fblocks = (int)(((long long)c->nnz * c->batch + 255) / 256);
    if (a.fblocks == 0) return DGSEM_OK;
  } else {
    a.R = R; a.rstride = c->rstride; a.rw = c->d_rw; a.roff = c->d_roff; a.rnn = c->d_rnn;
    a.p = static_cast<const T*>(c->Y);
    a.traces = traces; a.tbs = tbs; a.trs = trs;
    a.n = 0; a.step = c->d_step; a.done = c->d_done;
  }
  HexTimer t(c, s, DGHEX_K_TAIL);
  HCUDA(hex::launch_hex_tail<T>(a, s));
  return DGSEM_OK;
}

// One step of Algorithm 1: PMUT (p^n, drive of step n) -> q''^{n+1}; forcing
// rows of q''^{n+1}; K p^{n+1}; v^{n+3/2} = v^{n+1/2} + dt M^-1 (f - K p^{n+1}
// - C v^{n+1/2}), p^{n+2} = p^{n+1} + dt v^{n+3/2} into X; receivers of
// p^{n+1}; swap.
template <typename T>
int launch_step(dghex_ctx* c, cudaStream_t s, const double* drive, long long dbs, long long dks, int R, double* traces,
                long long tbs, long long trs) {
  if (c->K > 0) {
    PmutArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.B = c->batch; a.K = c->K; a.M = c->M;
    a.fp_ptr = c->d_fp_ptr; a.fp_off = c->d_fp_offB; a.Bm = c->d_Bm;
    a.p_prev = static_cast<const T*>(c->X);
    a.bsp = 1;
    const long long kmB = (long long)c->batch * c->K * c->M;
    a.q = c->q_state; a.qd = c->q_state + kmB; a.qdd = c->q_state + 2 * kmB;
    const long long km = (long long)c->K * c->M;
    a.omega2 = c->d_modal; a.twozw = c->d_modal + km; a.inv_mu = c->d_modal + 2 * km; a.eta = c->d_modal + 3 * km;
    a.drive = drive; a.dbs = dbs; a.dks = dks; a.n = 0; a.step = c->d_step; a.dt = c->dt;
    if (c->rx_switch >= 0) {
      a.rx_gain = c->d_rx_gain; a.rx_switch = c->rx_switch; a.step_base = c->d_step_base;
      a.volt = c->d_volt; a.vbs = (long long)c->K * dks; a.vks = dks;
    }
    HexTimer t(c, s, DGHEX_K_PMUT);
    HCUDA(launch_pmut_recv<T>(a, s));
  }
  int rc;
  if (c->K > 0 && (rc = launch_tail<T>(c, s, true, 0, nullptr, 0, 0))) return rc;
  if ((rc = launch_residual<T>(c, s, c->Y))) return rc;
  for (int d = 0; d < c->nd && c->has_pml; ++d) {
    const HexDom& D = c->dom[d];
    if (D.pml_elem.empty()) continue;
    const bool f = std::is_same<T, float>::value;
    hex::HexPmlArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.p = static_cast<const T*>(c->Y); a.psi = static_cast<const T*>(c->Psi); a.phi = static_cast<T*>(D.Phi);
    a.S = static_cast<T*>(c->S); a.Bp = c->Bp;
    a.elem = D.d_pml_elem; a.conn = D.d_conn;
    a.geo = f ? reinterpret_cast<const T*>(D.d_pml_geo32) : reinterpret_cast<const T*>(D.d_pml_geo64);
    a.zeta = f ? reinterpret_cast<const T*>(c->d_zeta32) : reinterpret_cast<const T*>(c->d_zeta64);
    a.ndof = c->ndof; a.slot_base = D.pslot0; a.npml = (int)D.pml_elem.size();
    a.c2 = T(D.c * D.c); a.dt = T(c->dt);
    for (int i = 0; i < D.n; ++i)
      for (int j = 0; j < D.n; ++j) a.D[i][j] = T(D.basis->D[i * D.n + j]);
    HexTimer t(c, s, DGHEX_K_PML);
    HCUDA(hex::launch_hex_pml<T>(a, D.n, s));
  }
  if ((rc = launch_update<T>(c, s, -c->dt, c->dt, c->Y, c->X, 2))) return rc;
  if ((rc = launch_tail<T>(c, s, false, R, traces, tbs, trs))) return rc;
  std::swap(c->X, c->Y);
  return DGSEM_OK;
}

// one FP64 field broadcast to every batch member (padding members stay 0)
template <typename T>
int upload_field(const std::vector<double>& h, void* dst, int batch, int Bp, long long ndof, cudaStream_t s) {
  std::vector<T> t((size_t)ndof * Bp, T(0));
  for (long long j = 0; j < ndof; ++j)
    for (int b = 0; b < batch; ++b) t[(size_t)j * Bp + b] = T(h[j]);
  HCUDA(cudaMemcpyAsync(dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  HCUDA(cudaStreamSynchronize(s));
  return DGSEM_OK;
}

template <typename T>
int run_impl(dghex_ctx* c, int nsteps, const double* drive, int R, double* traces_out, int flags, cudaStream_t s) {
  const bool fresh = !(flags & DGSEM_RUN_CONTINUE) || !c->state_valid;
  const size_t es = sizeof(T);
  if (fresh) c->steps_done = 0;
  HCUDA(cudaMemcpyAsync(c->d_step_base, &c->steps_done, sizeof(long long), cudaMemcpyHostToDevice, s));
  c->volt_n = 0;
  if (c->rx_switch >= 0 && c->K > 0) {
    const size_t nv = (size_t)c->batch * c->K * nsteps;
    if (nv > c->volt_cap) {
      dfree(c->d_volt);
      int rc = dmalloc(&c->d_volt, nv * sizeof(double));
      if (rc) return rc;
      c->volt_cap = nv;
    }
    c->volt_n = (long long)nv;
  }
  if (fresh) {
    HCUDA(cudaMemsetAsync(c->X, 0, es * c->Bp * c->ndof, s));
    HCUDA(cudaMemsetAsync(c->Y, 0, es * c->Bp * c->ndof, s));
    HCUDA(cudaMemsetAsync(c->V, 0, es * c->Bp * c->ndof, s));
    HCUDA(cudaMemsetAsync(c->S, 0, es * c->Bp * c->nslot, s));
    if (c->q_state) HCUDA(cudaMemsetAsync(c->q_state, 0, sizeof(double) * 3 * (size_t)c->batch * c->K * c->M, s));
    if (c->Psi) HCUDA(cudaMemsetAsync(c->Psi, 0, es * c->Bp * c->ndof, s));
    for (int d = 0; d < c->nd; ++d)
      if (c->dom[d].Phi)
        HCUDA(cudaMemsetAsync(c->dom[d].Phi, 0, es * c->Bp * 3 * c->dom[d].nl * c->dom[d].pml_elem.size(), s));
    if (c->has_init) {
      int rc;
      if (!c->init_p.empty() && (rc = upload_field<T>(c->init_p, c->X, c->batch, c->Bp, c->ndof, s))) return rc;
      if (!c->init_v.empty() && (rc = upload_field<T>(c->init_v, c->V, c->batch, c->Bp, c->ndof, s))) return rc;
      // v^{1/2} = p'^0 + dt/2 p''^0 with p''^0 = M^-1 (-K p^0 - C p'^0) (no forcing at rest),
      // p^1 = p^0 + dt v^{1/2}
      if ((rc = launch_residual<T>(c, s, c->X)) || (rc = launch_update<T>(c, s, -0.5 * c->dt, c->dt, c->X, c->Y, 1)))
        return rc;
    }
  }
  const double* d_drive = drive;
  const size_t dn = (size_t)c->batch * c->K * nsteps;
  if (c->K > 0) {
    if (!drive) return hfail(DGSEM_EINVAL, "drive is NULL with %d PMUTs", c->K);
    if (!is_device_ptr(drive)) {
      if (dn > c->drive_cap) {
        dfree(c->d_drive);
        int rc = dmalloc(&c->d_drive, dn * sizeof(double));
        if (rc) return rc;
        c->drive_cap = dn;
      }
      HCUDA(cudaMemcpyAsync(c->d_drive, drive, dn * sizeof(double), cudaMemcpyHostToDevice, s));
      d_drive = c->d_drive;
    }
  }
  double* d_traces = traces_out;
  const size_t tn = (size_t)c->batch * R * nsteps;
  const bool host_traces = R > 0 && !is_device_ptr(traces_out);
  if (host_traces) {
    if (tn > c->traces_cap) {
      dfree(c->d_traces);
      int rc = dmalloc(&c->d_traces, tn * sizeof(double));
      if (rc) return rc;
      c->traces_cap = tn;
    }
    d_traces = c->d_traces;
  }
  HCUDA(cudaMemsetAsync(c->d_step, 0, sizeof(int), s));
  HCUDA(cudaMemsetAsync(c->d_done, 0, sizeof(unsigned), s));
  for (int n = 0; n < nsteps; ++n) {
    int rc = launch_step<T>(c, s, d_drive, (long long)c->K * nsteps, nsteps, R, d_traces, (long long)R * nsteps, nsteps);
    if (rc) return rc;
  }
  // divergence check: receiver traces (they sample p every step) and the PMUT state
  HCUDA(cudaMemsetAsync(c->d_nf, 0, sizeof(int), s));
  if (R > 0) HCUDA(launch_nonfinite(d_traces, tn, c->d_nf, s));
  if (c->q_state) HCUDA(launch_nonfinite(c->q_state, (size_t)3 * c->batch * c->K * c->M, c->d_nf, s));
  if (host_traces) HCUDA(cudaMemcpyAsync(traces_out, d_traces, tn * sizeof(double), cudaMemcpyDeviceToHost, s));
  HCUDA(cudaStreamSynchronize(s));
  if (c->profiling) collect_timings(c);
  else c->ev_used.clear();
  int nf = 0;
  HCUDA(cudaMemcpy(&nf, c->d_nf, sizeof(int), cudaMemcpyDeviceToHost));
  if (nf) {
    c->state_valid = false;
    return hfail(DGSEM_EUNSTABLE, "non-finite receiver traces or PMUT state: the time step diverged (dt above the stability limit?)");
  }
  c->state_valid = true;
  c->steps_done += nsteps;
  return DGSEM_OK;
}

template <typename T>
int autotune_impl(dghex_ctx* c, int reps, int* chosen, cudaStream_t s) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  HCUDA(cudaMemsetAsync(c->Y, 0, sizeof(T) * (size_t)c->Bp * c->ndof, s));
  cudaEvent_t e0, e1;
  HCUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return hfail(DGSEM_ECUDA, "cudaEventCreate failed");
  }
  int rc = DGSEM_OK;
  for (int d = 0; d < c->nd && rc == DGSEM_OK; ++d) {
    const hex::HexVolArgs<T> a = vol_args<T>(c, d, c->Y);
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < hex::kHexVolVariants; ++v) {
      cudaError_t e = hex::launch_hex_vol<T>(a, c->dom[d].n, v, s);   // warm-up
      if (e != cudaSuccess) { rc = hfail(DGSEM_ECUDA, "autotune, variant %d: %s", v, cudaGetErrorString(e)); break; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = hex::launch_hex_vol<T>(a, c->dom[d].n, v, s);
      cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { rc = hfail(DGSEM_ECUDA, "autotune, variant %d: %s", v, cudaGetErrorString(e)); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = v; }
    }
    c->vol_variant[pi][d] = best;
    if (chosen) chosen[d] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" {

int dghex_mesh_create(const dghex_mesh_desc* d, dghex_ctx** out) {
  if (!out) return hfail(DGSEM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d || !d->domains) return hfail(DGSEM_EINVAL, "desc or domains is NULL");
  if (d->ndomains < 1 || d->ndomains > 2) return hfail(DGSEM_EINVAL, "ndomains must be 1 or 2");
  for (int k = 0; k < d->ndomains; ++k) {
    const dghex_domain_desc& D = d->domains[k];
    if (D.order < 1 || D.order > 8) return hfail(DGSEM_EINVAL, "domain %d: order must be 1..8", k);
    if (!(D.c > 0.0) || !(D.rho > 0.0)) return hfail(DGSEM_EINVAL, "domain %d: c and rho must be > 0", k);
    if (D.n_vert < 8 || D.n_elem < 1 || !D.vert || !D.elem) return hfail(DGSEM_EINVAL, "domain %d: empty mesh", k);
    for (long long i = 0; i < 8LL * D.n_elem; ++i)
      if (D.elem[i] < 0 || D.elem[i] >= D.n_vert)
        return hfail(DGSEM_EINVAL, "domain %d: element %lld lists vertex %d out of range", k, i / 8, D.elem[i]);
  }
  if (!(d->penalty_alpha > 0.0) && d->ndomains == 2) return hfail(DGSEM_EINVAL, "penalty_alpha must be > 0");
  if (d->dt <= 0.0 && !(d->cfl > 0.0)) return hfail(DGSEM_EINVAL, "cfl must be > 0 when dt is not given");
  auto check_faces = [&](int nf, const int* f, int dom, const char* what) -> int {
    if (nf < 0 || (nf > 0 && !f)) return hfail(DGSEM_EINVAL, "%s: bad list", what);
    for (int i = 0; i < nf; ++i)
      if (f[2 * i] < 0 || f[2 * i] >= d->domains[dom].n_elem || f[2 * i + 1] < 0 || f[2 * i + 1] > 5)
        return hfail(DGSEM_EINVAL, "%s: entry %d out of range", what, i);
    return DGSEM_OK;
  };
  int rc;
  if (d->ndomains == 2) {
    if (d->n_fine_faces < 1 || d->n_coarse_faces < 1) return hfail(DGSEM_EINVAL, "two domains need the interface face lists");
    if ((rc = check_faces(d->n_fine_faces, d->fine_faces, 0, "fine_faces")) ||
        (rc = check_faces(d->n_coarse_faces, d->coarse_faces, 1, "coarse_faces")))
      return rc;
  }
  if ((rc = check_faces(d->n_pmut_faces, d->pmut_faces, 0, "pmut_faces"))) return rc;
  dghex_ctx* c = new dghex_ctx();
  cudaGetDevice(&c->device);
  c->nd = d->ndomains;
  c->fcount.assign(c->nd, {});
  auto& fcount = c->fcount;
  long long node0 = 0, vslot = 0;
  for (int k = 0; k < c->nd; ++k) {
    const dghex_domain_desc& S = d->domains[k];
    HexDom& D = c->dom[k];
    D.N = S.order; D.n = S.order + 1; D.nl = D.n * D.n * D.n;
    D.ne = S.n_elem; D.nv = S.n_vert; D.c = S.c; D.rho = S.rho;
    D.vert.assign(S.vert, S.vert + 3 * (size_t)S.n_vert);
    D.elem.assign(S.elem, S.elem + 8 * (size_t)S.n_elem);
    D.basis = new dgtab::Basis1D(D.N);
    number_nodes(D, node0, fcount[k]);
    node0 += D.nnode;
    D.vslot0 = vslot;
    vslot += (long long)D.ne * D.nl;
  }
  c->ndof = node0;
  c->nvol = vslot;
  if (c->ndof >= (1LL << 31) || c->nvol >= (1LL << 31)) {
    dghex_destroy(c);
    return hfail(DGSEM_EINVAL, "mesh too large (%lld nodes, %lld element nodes)", node0, vslot);
  }
  // listed faces must be boundary faces of their domain
  auto boundary = [&](int dom, int nf, const int* f, const char* what) -> int {
    const HexDom& D = c->dom[dom];
    for (int i = 0; i < nf; ++i) {
      const int e = f[2 * i], lf = f[2 * i + 1], ax = lf >> 1, side = lf & 1;
      std::array<int, 4> key;
      int k = 0;
      for (int cc = 0; cc < 8; ++cc)
        if (((cc >> ax) & 1) == side) key[k++] = D.elem[(size_t)e * 8 + cc];
      std::sort(key.begin(), key.end());
      if (fcount[dom][key] != 1) return hfail(DGSEM_EINVAL, "%s: entry %d is not a boundary face", what, i);
    }
    return DGSEM_OK;
  };
  if ((c->nd == 2 && ((rc = boundary(0, d->n_fine_faces, d->fine_faces, "fine_faces")) ||
                      (rc = boundary(1, d->n_coarse_faces, d->coarse_faces, "coarse_faces")))) ||
      (rc = boundary(0, d->n_pmut_faces, d->pmut_faces, "pmut_faces"))) {
    dghex_destroy(c);
    return rc;
  }
  // node positions (host)
  c->xyz.assign(3 * (size_t)c->ndof, 0.0);
  for (int k = 0; k < c->nd; ++k) {
    const HexDom& D = c->dom[k];
    for (int e = 0; e < D.ne; ++e) {
      double V[24];
      elem_verts(D, e, V);
      for (int i = 0; i < D.nl; ++i) {
        const double r[3] = {D.basis->x[i % D.n], D.basis->x[(i / D.n) % D.n], D.basis->x[i / (D.n * D.n)]};
        double x[3], J[3][3];
        hex::tri_map(V, r, x, J);
        const long long id = D.conn[(size_t)e * D.nl + i];
        for (int a = 0; a < 3; ++a) c->xyz[3 * id + a] = x[a];
      }
    }
  }
  // geometry on the device
  int* d_bad = nullptr;
  rc = dmalloc(&c->d_Mloc, sizeof(double) * c->nvol);
  if (!rc) rc = dmalloc(&d_bad, sizeof(int));
  if (!rc && cudaMemset(d_bad, 0, sizeof(int)) != cudaSuccess) rc = hfail(DGSEM_ECUDA, "memset");
  for (int k = 0; k < c->nd && !rc; ++k) {
    HexDom& D = c->dom[k];
    if ((rc = upload(&D.d_vert, D.vert)) || (rc = upload(&D.d_elem, D.elem)) || (rc = upload(&D.d_conn, D.conn)) ||
        (rc = dmalloc(&D.d_G64, sizeof(double) * 6 * (size_t)D.ne * hex::gstride(D.n))) ||
        (rc = dmalloc(&D.d_G32, sizeof(float) * 6 * (size_t)D.ne * hex::gstride(D.n))))
      break;
    hex::GeomArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vert = D.d_vert; a.elem = D.d_elem; a.ne = D.ne; a.n = D.n;
    for (int i = 0; i < D.n; ++i) { a.xi[i] = D.basis->x[i]; a.w[i] = D.basis->w[i]; }
    a.c2 = D.c * D.c;
    a.G64 = D.d_G64; a.G32 = D.d_G32; a.Mloc = c->d_Mloc + D.vslot0; a.bad = d_bad;
    const cudaError_t e = hex::launch_geom(a, 0);
    if (e != cudaSuccess) rc = hfail(DGSEM_ECUDA, "geometry kernel: %s", cudaGetErrorString(e));
  }
  int bad = 0;
  if (!rc && cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = hfail(DGSEM_ECUDA, "geometry kernel failed");
  dfree(d_bad);
  if (!rc && bad > 0) rc = hfail(DGSEM_EINVAL, "%d GLL nodes with a non-positive Jacobian", bad);
  if (rc) {
    dghex_destroy(c);
    return rc;
  }
  // time step: CFL on the shortest element edge
  double hmin_t = 1e300, cmax = 0.0;
  static const int edges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
  for (int k = 0; k < c->nd; ++k) {
    const HexDom& D = c->dom[k];
    double gap = 1e300;
    for (int i = 0; i < D.N; ++i) gap = std::min(gap, D.basis->x[i + 1] - D.basis->x[i]);
    for (int e = 0; e < D.ne; ++e) {
      double V[24];
      elem_verts(D, e, V);
      double h = 1e300;
      for (auto& ed : edges) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (V[3 * ed[0] + a] - V[3 * ed[1] + a]) * (V[3 * ed[0] + a] - V[3 * ed[1] + a]);
        h = std::min(h, std::sqrt(s));
      }
      hmin_t = std::min(hmin_t, h / 2.0 * gap);
    }
    cmax = std::max(cmax, D.c);
  }
  c->dt_cfl = d->dt > 0.0 ? d->dt : d->cfl * hmin_t / cmax;
  c->dt_fixed = d->dt > 0.0;
  c->dt = c->dt_cfl;
  if (c->nd == 2 && (rc = setup_interface(c, d))) {
    dghex_destroy(c);
    return rc;
  }
  std::vector<int> pf(d->pmut_faces, d->pmut_faces + 2 * (size_t)std::max(0, d->n_pmut_faces));
  c->pmut_faces = pf;
  setup_pmut_nodes(c, pf);
  if ((rc = build_slots(c)) || (rc = dmalloc(&c->d_M, sizeof(double) * c->ndof)) ||
      (rc = dmalloc(&c->d_Minv64, sizeof(double) * c->ndof)) || (rc = dmalloc(&c->d_Minv32, sizeof(float) * c->ndof)) ||
      (rc = dmalloc(&c->d_step, sizeof(int))) || (rc = dmalloc(&c->d_done, sizeof(unsigned))) ||
      (rc = dmalloc(&c->d_nf, sizeof(int)))) {
    dghex_destroy(c);
    return rc;
  }
  cudaError_t e = hex::launch_mass(c->d_Mloc, c->d_node_ptr, c->d_node_slot, c->nvol, c->ndof, c->d_Minv64, c->d_Minv32,
                                   c->d_M, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    c->Mh.resize((size_t)c->ndof);
    e = cudaMemcpy(c->Mh.data(), c->d_M, sizeof(double) * c->ndof, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c->d_step_base), sizeof(long long));
  if (e != cudaSuccess) {
    dghex_destroy(c);
    return hfail(DGSEM_ECUDA, "mass kernel: %s", cudaGetErrorString(e));
  }
  *out = c;
  return DGSEM_OK;
}

int dghex_get_dt(const dghex_ctx* c, double* dt, long long* ndof) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (dt) *dt = c->dt;
  if (ndof) *ndof = c->ndof;
  return DGSEM_OK;
}

int dghex_nodes(const dghex_ctx* c, long long* ndof, long long* first_secondary, const double** xyz) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (ndof) *ndof = c->ndof;
  if (first_secondary) *first_secondary = c->nd == 2 ? c->dom[1].node0 : c->ndof;
  if (xyz) *xyz = c->xyz.data();
  return DGSEM_OK;
}

int dghex_pmut_nodes(const dghex_ctx* c, int* n, const double** xyz, const double** weight) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (n) *n = (int)c->pn_id.size();
  if (xyz) *xyz = c->pn_xyz.data();
  if (weight) *weight = c->pn_w.data();
  return DGSEM_OK;
}

int dghex_pmut_set(dghex_ctx* c, int K, int M, const int* foot_ptr, const int* foot_node, const double* shape_un,
                   const double* freq_hz, const double* damping, const double* eta, const double* modal_mass) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (K < 0 || M < 1 || M > DG_MAXM) return hfail(DGSEM_EINVAL, "n_pmut >= 0 and 1 <= n_modes <= %d", DG_MAXM);
  if (K > 0 && (!foot_ptr || !freq_hz || !damping || !eta)) return hfail(DGSEM_EINVAL, "NULL PMUT array");
  const int npn = (int)c->pn_id.size();
  std::vector<int> fp_ptr(foot_ptr, foot_ptr + (K > 0 ? K + 1 : 0));
  if (K > 0 && fp_ptr[0] != 0) return hfail(DGSEM_EINVAL, "foot_ptr[0] must be 0");
  for (int k = 0; k < K; ++k)
    if (fp_ptr[k + 1] < fp_ptr[k]) return hfail(DGSEM_EINVAL, "foot_ptr must be non-decreasing");
  const int nnz = K > 0 ? fp_ptr[K] : 0;
  if (nnz > 0 && (!foot_node || !shape_un)) return hfail(DGSEM_EINVAL, "NULL footprint");
  std::vector<long long> off(nnz);
  std::vector<double> B((size_t)nnz * M);
  std::vector<int> entk(nnz);
  for (int k = 0; k < K; ++k)
    for (int e = fp_ptr[k]; e < fp_ptr[k + 1]; ++e) {
      const int j = foot_node[e];
      if (j < 0 || j >= npn) return hfail(DGSEM_EINVAL, "foot_node[%d] = %d out of range", e, j);
      off[e] = c->pn_id[j];
      entk[e] = k;
      for (int m = 0; m < M; ++m) B[(size_t)e * M + m] = c->pn_w[j] * shape_un[(size_t)e * M + m];
    }
  std::vector<double> modal(4 * (size_t)K * M);
  const size_t km = (size_t)K * M;
  for (size_t i = 0; i < km; ++i) {
    const double w = 2.0 * M_PI * freq_hz[i];
    const double mu = modal_mass ? modal_mass[i] : 1.0;
    if (!(mu > 0.0)) return hfail(DGSEM_EINVAL, "modal_mass must be > 0");
    modal[i] = w * w;
    modal[km + i] = 2.0 * damping[i] * w;
    modal[2 * km + i] = 1.0 / mu;
    modal[3 * km + i] = eta[i];
  }
  dfree(c->d_fp_ptr); dfree(c->d_fp_off); dfree(c->d_Bm); dfree(c->d_ent_k); dfree(c->d_modal);
  c->K = K; c->M = M; c->nnz = nnz;
  c->ent_node = off;
  c->kappa = c->dom[0].rho * c->dom[0].c * c->dom[0].c;
  int rc;
  if ((rc = upload(&c->d_fp_ptr, fp_ptr)) || (rc = upload(&c->d_fp_off, off)) || (rc = upload(&c->d_Bm, B)) ||
      (rc = upload(&c->d_ent_k, entk)) || (rc = upload(&c->d_modal, modal)))
    return rc;
  return build_slots(c);
}

int dghex_get_matches(const dghex_ctx* c, int* q, int* coarse_face, double* ref, long long n) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (q) *q = c->q;
  const long long have = (long long)c->match.size();
  if ((coarse_face || ref) && n < have) return hfail(DGSEM_EINVAL, "arrays hold %lld points, %lld needed", n, have);
  if (coarse_face) std::copy(c->match.begin(), c->match.end(), coarse_face);
  if (ref) std::copy(c->refm.begin(), c->refm.end(), ref);
  return DGSEM_OK;
}

int dghex_set_state(dghex_ctx* c, const double* p0, const double* v0) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  c->init_p.clear();
  c->init_v.clear();
  if (p0) c->init_p.assign(p0, p0 + c->ndof);
  if (v0) c->init_v.assign(v0, v0 + c->ndof);
  c->has_init = p0 || v0;
  c->state_valid = false;
  return DGSEM_OK;
}

int dghex_run(dghex_ctx* c, int precision, int batch, int nsteps, const double* drive, int n_recv, const double* recv_xyz,
              double* traces, int flags, void* stream) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return hfail(DGSEM_EINVAL, "bad precision");
  if (batch < 1 || nsteps < 0 || n_recv < 0) return hfail(DGSEM_EINVAL, "batch >= 1, nsteps >= 0, n_recv >= 0");
  if (n_recv > 0 && (!recv_xyz || !traces)) return hfail(DGSEM_EINVAL, "receivers without positions or traces");
  if ((flags & DGSEM_RUN_CONTINUE) && (!c->state_valid || c->prec != precision || c->batch != batch))
    return hfail(DGSEM_ESTATE, "DGSEM_RUN_CONTINUE needs a valid state from a run (or a loaded checkpoint) "
                               "with the same precision and batch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_run_state(c, precision, batch);
  if (rc) return rc;
  if ((rc = setup_receivers(c, n_recv, recv_xyz))) return rc;
  // a run that fails part-way leaves no state to continue from
  rc = precision == DGSEM_FP32_MIXED ? run_impl<float>(c, nsteps, drive, n_recv, traces, flags, s)
                                     : run_impl<double>(c, nsteps, drive, n_recv, traces, flags, s);
  if (rc != DGSEM_OK) c->state_valid = false;
  return rc;
}

int dghex_get_pressure(const dghex_ctx* c, double* p, size_t len) {
  if (!c || !p) return hfail(DGSEM_EINVAL, "NULL argument");
  if (!c->state_valid) return hfail(DGSEM_ESTATE, "no run yet");
  const size_t n = (size_t)c->batch * c->ndof, nb = (size_t)c->Bp * c->ndof;
  if (len < n) return hfail(DGSEM_EINVAL, "p holds %zu values, %zu needed", len, n);
  std::vector<double> t(nb);
  if (c->prec == DGSEM_FP32_MIXED) {
    std::vector<float> f(nb);
    HCUDA(cudaMemcpy(f.data(), c->X, nb * sizeof(float), cudaMemcpyDeviceToHost));
    std::copy(f.begin(), f.end(), t.begin());
  } else {
    HCUDA(cudaMemcpy(t.data(), c->X, nb * sizeof(double), cudaMemcpyDeviceToHost));
  }
  for (int b = 0; b < c->batch; ++b)
    for (long long j = 0; j < c->ndof; ++j) p[(size_t)b * c->ndof + j] = t[(size_t)j * c->Bp + b];
  return DGSEM_OK;
}

namespace {
// C_jj / M_jj of every domain's absorbing faces (Nanson-weighted GLL
// collocation of the damping form of eq. Wf_4), uploaded in both precisions;
// dt held to 1 / max of it.
int apply_absorbing(dghex_ctx* c, const std::vector<double>* alpha) {
  dfree(c->d_damp64);
  dfree(c->d_damp32);
  std::vector<double> C((size_t)c->ndof, 0.0);
  bool any = false;
  for (int d = 0; d < c->nd; ++d) {
    const HexDom& D = c->dom[d];
    const auto& fl = c->abs_faces[d];
    for (size_t k = 0; k < fl.size() / 2; ++k) {
      const int e = fl[2 * k], f = fl[2 * k + 1];
      double V[24];
      elem_verts(D, e, V);
      const int ax = f >> 1, fixed = (f & 1) ? D.N : 0;
      const int t0 = ax == 0 ? 1 : 0, t1 = ax == 2 ? 1 : 2;
      for (int i = 0; i < D.nl; ++i) {
        const int l[3] = {i % D.n, (i / D.n) % D.n, i / (D.n * D.n)};
        if (l[ax] != fixed) continue;
        const double r[3] = {D.basis->x[l[0]], D.basis->x[l[1]], D.basis->x[l[2]]};
        double x[3], J[3][3], nrm[3];
        hex::tri_map(V, r, x, J);
        const double dS = hex::face_normal(f, J, nrm);
        C[D.conn[(size_t)e * D.nl + i]] += D.c * D.basis->w[l[t0]] * D.basis->w[l[t1]] * dS;
        any = true;
      }
    }
  }
  c->dt = c->dt_cfl;
  c->state_valid = false;
  if (alpha) any = true;
  if (!any) return DGSEM_OK;
  double smax = 0.0;
  std::vector<float> s32((size_t)c->ndof);
  for (long long j = 0; j < c->ndof; ++j) {
    C[j] /= c->Mh[j];
    if (alpha) C[j] += (*alpha)[j];
    smax = std::max(smax, C[j]);
    s32[j] = (float)C[j];
  }
  if (c->dt_fixed && c->dt > 1.0 / smax)
    return hfail(DGSEM_EUNSTABLE, "dt %.4g above the damping limit 1 / max (C/M + alpha) = %.4g", c->dt, 1.0 / smax);
  if (!c->dt_fixed) c->dt = std::min(c->dt, 1.0 / smax);
  int rc;
  if ((rc = upload(&c->d_damp64, C)) || (rc = upload(&c->d_damp32, s32))) return rc;
  return DGSEM_OK;
}

// Layer profiles zeta_d (Sec. 2: zeta~ (s - sin(2 pi s) / (2 pi)), zeta~ =
// c / l log(1/R), s the depth into a layer of thickness l measured from the
// side of the domain's bounding box), the layer elements (any node with a
// non-zero profile), their J^-1 and w |J| at the GLL nodes, the node
// coefficients, the layer slots and the damping limit of dt.
int rebuild_pml(dghex_ctx* c) {
  std::vector<double> zeta(3 * (size_t)c->ndof, 0.0);
  for (int d = 0; d < c->nd; ++d) {
    HexDom& D = c->dom[d];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < D.nv; ++v)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], D.vert[3 * (size_t)v + a]);
        hi[a] = std::max(hi[a], D.vert[3 * (size_t)v + a]);
      }
    for (int side = 0; side < 6; ++side) {
      const double t = D.pml_th[side];
      if (!(t > 0.0)) continue;
      const int ax = side >> 1;
      const double zt = D.c / t * std::log(1.0 / c->pml_R);
      for (long long j = D.node0; j < D.node0 + D.nnode; ++j) {
        const double x = c->xyz[3 * j + ax];
        double sd = (side & 1) ? (x - (hi[ax] - t)) / t : (lo[ax] + t - x) / t;
        sd = std::min(1.0, std::max(0.0, sd));
        zeta[(size_t)ax * c->ndof + j] += zt * (sd - std::sin(2.0 * M_PI * sd) / (2.0 * M_PI));
      }
    }
  }
  c->has_pml = false;
  for (double z : zeta) c->has_pml = c->has_pml || z != 0.0;
  dfree(c->d_zeta64); dfree(c->d_zeta32); dfree(c->d_beta64); dfree(c->d_beta32);
  dfree(c->d_gamma64); dfree(c->d_gamma32);
  c->pml_alpha.clear();
  for (int d = 0; d < c->nd; ++d) {
    HexDom& D = c->dom[d];
    D.pml_elem.clear();
    dfree(D.d_pml_elem); dfree(D.d_pml_geo64); dfree(D.d_pml_geo32);
    if (!c->has_pml) continue;
    for (int e = 0; e < D.ne; ++e) {
      bool in = false;
      for (int i = 0; i < D.nl && !in; ++i) {
        const int j = D.conn[(size_t)e * D.nl + i];
        in = zeta[j] != 0.0 || zeta[c->ndof + j] != 0.0 || zeta[2 * c->ndof + j] != 0.0;
      }
      if (in) D.pml_elem.push_back(e);
    }
    std::vector<double> geo(D.pml_elem.size() * 10 * (size_t)D.nl);
    for (size_t k = 0; k < D.pml_elem.size(); ++k) {
      double V[24];
      elem_verts(D, D.pml_elem[k], V);
      for (int i = 0; i < D.nl; ++i) {
        const int l[3] = {i % D.n, (i / D.n) % D.n, i / (D.n * D.n)};
        const double r[3] = {D.basis->x[l[0]], D.basis->x[l[1]], D.basis->x[l[2]]};
        double x[3], J[3][3], Ji[3][3];
        hex::tri_map(V, r, x, J);
        const double det = hex::inv3(J, Ji);
        double* g = &geo[k * 10 * D.nl + i];
        for (int q = 0; q < 9; ++q) g[(size_t)q * D.nl] = Ji[q / 3][q % 3];
        g[9 * (size_t)D.nl] = D.basis->w[l[0]] * D.basis->w[l[1]] * D.basis->w[l[2]] * det;
      }
    }
    std::vector<float> g32(geo.begin(), geo.end());
    int rc;
    if ((rc = upload(&D.d_pml_elem, D.pml_elem)) || (rc = upload(&D.d_pml_geo64, geo)) || (rc = upload(&D.d_pml_geo32, g32)))
      return rc;
  }
  if (c->has_pml) {
    const size_t n = (size_t)c->ndof;
    std::vector<double> beta(n), gamma(n);
    c->pml_alpha.resize(n);
    for (size_t j = 0; j < n; ++j) {
      const double z1 = zeta[j], z2 = zeta[n + j], z3 = zeta[2 * n + j];
      c->pml_alpha[j] = z1 + z2 + z3;
      beta[j] = z1 * z2 + z2 * z3 + z3 * z1;
      gamma[j] = z1 * z2 * z3;
    }
    std::vector<float> z32(zeta.begin(), zeta.end()), b32(beta.begin(), beta.end()), g32(gamma.begin(), gamma.end());
    int rc;
    if ((rc = upload(&c->d_zeta64, zeta)) || (rc = upload(&c->d_zeta32, z32)) || (rc = upload(&c->d_beta64, beta)) ||
        (rc = upload(&c->d_beta32, b32)) || (rc = upload(&c->d_gamma64, gamma)) || (rc = upload(&c->d_gamma32, g32)))
      return rc;
  }
  int rc = build_slots(c);
  if (rc) return rc;
  return apply_absorbing(c, c->has_pml ? &c->pml_alpha : nullptr);
}

bool face_in(const std::vector<int>& list, int e, int f) {
  for (size_t k = 0; k < list.size() / 2; ++k)
    if (list[2 * k] == e && list[2 * k + 1] == f) return true;
  return false;
}

struct HexCkpt {
  char magic[8];
  int prec, batch, Bp, K, M, nnz;
  long long ndof, steps;
};
}  // namespace

int dghex_set_absorbing_faces(dghex_ctx* c, int domain, int n, const int* faces) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (domain < 0 || domain >= c->nd) return hfail(DGSEM_EINVAL, "domain %d out of range", domain);
  if (n < 0 || (n > 0 && !faces)) return hfail(DGSEM_EINVAL, "bad face list");
  const HexDom& D = c->dom[domain];
  std::vector<int> fl(faces, faces + 2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const int e = fl[2 * i], f = fl[2 * i + 1];
    if (e < 0 || e >= D.ne || f < 0 || f > 5) return hfail(DGSEM_EINVAL, "face entry %d out of range", i);
    std::array<int, 4> key;
    int k = 0;
    for (int cc = 0; cc < 8; ++cc)
      if (((cc >> (f >> 1)) & 1) == (f & 1)) key[k++] = D.elem[(size_t)e * 8 + cc];
    std::sort(key.begin(), key.end());
    auto it = c->fcount[domain].find(key);
    if (it == c->fcount[domain].end() || it->second != 1) return hfail(DGSEM_EINVAL, "face entry %d is not a boundary face", i);
    if ((domain == 0 && (face_in(c->ff, e, f) || face_in(c->pmut_faces, e, f))) || (domain == 1 && face_in(c->cf, e, f)))
      return hfail(DGSEM_EINVAL, "face entry %d lies on the interface or on Gamma_PMUT", i);
  }
  c->abs_faces[domain] = fl;
  return apply_absorbing(c, c->has_pml ? &c->pml_alpha : nullptr);
}

int dghex_set_pml(dghex_ctx* c, int domain, const double* thickness, double R) {
  if (!c || !thickness) return hfail(DGSEM_EINVAL, "NULL argument");
  if (domain < 0 || domain >= c->nd) return hfail(DGSEM_EINVAL, "domain %d out of range", domain);
  if (!(R > 0.0 && R < 1.0)) return hfail(DGSEM_EINVAL, "R must lie in (0, 1)");
  for (int k = 0; k < 6; ++k)
    if (!(thickness[k] >= 0.0) || !std::isfinite(thickness[k])) return hfail(DGSEM_EINVAL, "thickness[%d] must be >= 0", k);
  for (int k = 0; k < 6; ++k) c->dom[domain].pml_th[k] = thickness[k];
  c->pml_R = R;
  return rebuild_pml(c);
}

int dghex_pmut_set_receive(dghex_ctx* c, long long n_switch, const double* capacitance, int sign) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (n_switch < 0) {
    c->rx_switch = -1;
    return DGSEM_OK;
  }
  if (c->K == 0) return hfail(DGSEM_ESTATE, "no PMUT array: call dghex_pmut_set first");
  if (!capacitance) return hfail(DGSEM_EINVAL, "NULL capacitance");
  if (sign != 1 && sign != -1) return hfail(DGSEM_EINVAL, "sign must be +1 or -1");
  std::vector<double> gain(c->K);
  for (int k = 0; k < c->K; ++k) {
    if (!(capacitance[k] > 0.0) || !std::isfinite(capacitance[k]))
      return hfail(DGSEM_EINVAL, "capacitance[%d] must be > 0", k);
    gain[k] = sign / capacitance[k];
  }
  dfree(c->d_rx_gain);
  int rc = upload(&c->d_rx_gain, gain);
  if (rc) {
    c->rx_switch = -1;
    return rc;
  }
  c->rx_switch = n_switch;
  return DGSEM_OK;
}

int dghex_get_voltages(const dghex_ctx* c, double* out, size_t n) {
  if (!c || !out) return hfail(DGSEM_EINVAL, "NULL argument");
  if (c->volt_n == 0 || !c->d_volt) return hfail(DGSEM_ESTATE, "no voltage record: configure dghex_pmut_set_receive and run");
  if (n < (size_t)c->volt_n) return hfail(DGSEM_EINVAL, "buffer of %zu doubles is smaller than %lld", n, c->volt_n);
  HCUDA(cudaMemcpy(out, c->d_volt, (size_t)c->volt_n * sizeof(double), cudaMemcpyDeviceToHost));
  return DGSEM_OK;
}

int dghex_state_save(const dghex_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return hfail(DGSEM_EINVAL, "NULL argument");
  if (!c->state_valid) return hfail(DGSEM_ESTATE, "no state to save");
  if (c->has_pml) return hfail(DGSEM_ESTATE, "checkpoints of a state with a layer are not supported");
  const size_t es = c->prec == DGSEM_FP32_MIXED ? sizeof(float) : sizeof(double);
  const size_t field = (size_t)c->Bp * c->ndof * es;
  const size_t qb = (size_t)3 * c->batch * c->K * c->M * sizeof(double);
  const size_t need = sizeof(HexCkpt) + 3 * field + qb;
  if (!buf) {
    *len = need;
    return DGSEM_OK;
  }
  if (*len < need) return hfail(DGSEM_EINVAL, "buffer too small (%zu < %zu)", *len, need);
  HCUDA(cudaDeviceSynchronize());
  HexCkpt h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "DGHEXCK2", 8);
  h.prec = c->prec; h.batch = c->batch; h.Bp = c->Bp; h.K = c->K; h.M = c->M; h.nnz = c->nnz;
  h.ndof = c->ndof; h.steps = c->steps_done;
  unsigned char* o = static_cast<unsigned char*>(buf);
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  for (const void* src : {c->X, c->Y, c->V}) {
    HCUDA(cudaMemcpy(o, src, field, cudaMemcpyDeviceToHost));
    o += field;
  }
  if (qb) HCUDA(cudaMemcpy(o, c->q_state, qb, cudaMemcpyDeviceToHost));
  *len = need;
  return DGSEM_OK;
}

int dghex_state_load(dghex_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) return hfail(DGSEM_EINVAL, "NULL argument");
  if (len < sizeof(HexCkpt)) return hfail(DGSEM_EINVAL, "buffer too small");
  HexCkpt h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, "DGHEXCK2", 8) != 0) return hfail(DGSEM_EINVAL, "not a checkpoint of this library");
  if (h.ndof != c->ndof || h.K != c->K || h.M != c->M || h.nnz != c->nnz)
    return hfail(DGSEM_EINVAL, "checkpoint of another mesh or PMUT array");
  if (h.prec != DGSEM_FP64 && h.prec != DGSEM_FP32_MIXED) return hfail(DGSEM_EINVAL, "bad precision in checkpoint");
  int rc = ensure_run_state(c, h.prec, h.batch);
  if (rc) return rc;
  if (c->Bp != h.Bp) return hfail(DGSEM_EINVAL, "checkpoint batch layout differs");
  const size_t es = c->prec == DGSEM_FP32_MIXED ? sizeof(float) : sizeof(double);
  const size_t field = (size_t)c->Bp * c->ndof * es;
  const size_t qb = (size_t)3 * c->batch * c->K * c->M * sizeof(double);
  if (len < sizeof(HexCkpt) + 3 * field + qb) return hfail(DGSEM_EINVAL, "truncated checkpoint");
  const unsigned char* o = static_cast<const unsigned char*>(buf) + sizeof(HexCkpt);
  HCUDA(cudaMemset(c->S, 0, (size_t)c->Bp * c->nslot * es));
  for (void* dst : {c->X, c->Y, c->V}) {
    HCUDA(cudaMemcpy(dst, o, field, cudaMemcpyHostToDevice));
    o += field;
  }
  if (qb) HCUDA(cudaMemcpy(c->q_state, o, qb, cudaMemcpyHostToDevice));
  c->steps_done = h.steps;
  c->state_valid = true;
  return DGSEM_OK;
}

int dghex_energy(dghex_ctx* c, double* e, int n) {
  if (!c || !e) return hfail(DGSEM_EINVAL, "NULL argument");
  if (!c->state_valid) return hfail(DGSEM_ESTATE, "no state: run first");
  if (c->prec != DGSEM_FP64) return hfail(DGSEM_ESTATE, "the energy diagnostic needs an FP64 state");
  if (n < c->batch) return hfail(DGSEM_EINVAL, "e holds %d values, %d needed", n, c->batch);
  cudaStream_t s = 0;
  const size_t field = sizeof(double) * (size_t)c->Bp * c->ndof;
  double* w = nullptr;
  double* d_e = nullptr;
  int rc;
  if ((rc = dmalloc(&w, field)) || (rc = dmalloc(&d_e, sizeof(double) * c->batch))) {
    dfree(w);
    return rc;
  }
  // w = M^-1 K p^{n+1}: the stiffness and interface slots of Y gathered by the
  // update kernel into a zero field (forcing and layer slots cleared: K only)
  cudaError_t err = cudaMemsetAsync(w, 0, field, s);
  if (err == cudaSuccess && c->nslot > c->fslot0)
    err = cudaMemsetAsync(static_cast<double*>(c->S) + (size_t)c->fslot0 * c->Bp, 0,
                          sizeof(double) * (size_t)c->Bp * (c->nslot - c->fslot0), s);
  if (err == cudaSuccess) {
    const double* dsave = c->d_damp64;
    c->d_damp64 = nullptr;                  // K only: no damping on the (zero) scratch velocity
    rc = launch_residual<double>(c, s, c->Y);
    if (!rc) rc = launch_update<double>(c, s, 1.0, 0.0, c->Y, c->Y, 0, w);
    c->d_damp64 = const_cast<double*>(dsave);
    if (!rc) err = hex::launch_energy(c->d_M, static_cast<const double*>(c->V), static_cast<const double*>(c->X), w,
                                      c->ndof, c->batch, c->Bp, d_e, s);
  }
  if (!rc && err == cudaSuccess) err = cudaMemcpy(e, d_e, sizeof(double) * c->batch, cudaMemcpyDeviceToHost);
  dfree(w);
  dfree(d_e);
  if (rc) return rc;
  if (err != cudaSuccess) return hfail(DGSEM_ECUDA, "energy: %s", cudaGetErrorString(err));
  return DGSEM_OK;
}

int dghex_check_stability(dghex_ctx* c, int iters, double* lambda_max) {
  if (!c || iters < 1) return hfail(DGSEM_EINVAL, "ctx is NULL or iters < 1");
  int rc = ensure_run_state(c, DGSEM_FP64, 1);
  if (rc) return rc;
  c->state_valid = false;
  double* P = static_cast<double*>(c->Y);
  double* V = static_cast<double*>(c->V);
  double* d_n2 = nullptr;
  if ((rc = dmalloc(&d_n2, 2 * sizeof(double)))) return rc;
  // deterministic start vector in [-1, 1] (a 64-bit linear congruential sequence)
  std::vector<double> x((size_t)c->ndof);
  unsigned long long st = 0x9E3779B97F4A7C15ULL;
  for (auto& v : x) {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    v = (double)(st >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
  cudaStream_t s = 0;
  double lam = 0.0;
  cudaError_t e = cudaMemcpy(P, x.data(), x.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->S, 0, sizeof(double) * c->nslot, s);
  for (int it = 0; it < iters && e == cudaSuccess && rc == DGSEM_OK; ++it) {
    // v = M^-1 K x through the step's own kernels (zero forcing slots, v = 0 first)
    e = cudaMemsetAsync(V, 0, sizeof(double) * c->ndof, s);
    if (e != cudaSuccess) break;
    if ((rc = launch_residual<double>(c, s, P)) || (rc = launch_update<double>(c, s, 1.0, 0.0, P, P))) break;
    if ((e = hex::launch_norm2(P, c->ndof, d_n2, s)) != cudaSuccess) break;
    if ((e = hex::launch_norm2(V, c->ndof, d_n2 + 1, s)) != cudaSuccess) break;
    double n2[2];
    if ((e = cudaMemcpy(n2, d_n2, sizeof(n2), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    lam = std::sqrt(n2[1] / n2[0]);
    if (!(n2[1] > 0.0) || !std::isfinite(lam)) break;
    e = hex::launch_scale(P, V, d_n2 + 1, c->ndof, s);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  dfree(d_n2);
  if (rc) return rc;
  if (e != cudaSuccess) return hfail(DGSEM_ECUDA, "stability check: %s", cudaGetErrorString(e));
  if (lambda_max) *lambda_max = lam;
  if (lam > 0.0 && c->dt > 0.95 * 2.0 / std::sqrt(lam))
    return hfail(DGSEM_EUNSTABLE, "dt %.4g above 0.95 * 2 / sqrt(lambda_max) = %.4g", c->dt, 0.95 * 2.0 / std::sqrt(lam));
  return DGSEM_OK;
}

int dghex_set_interface_kernel(dghex_ctx* c, int general) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  c->force_general_iface = general != 0;
  return DGSEM_OK;
}

int dghex_num_volume_variants(const dghex_ctx* c, int* n) {
  if (!c || !n) return hfail(DGSEM_EINVAL, "NULL argument");
  *n = hex::kHexVolVariants;
  return DGSEM_OK;
}

int dghex_set_volume_variant(dghex_ctx* c, int precision, const int* variants) {
  if (!c || !variants) return hfail(DGSEM_EINVAL, "NULL argument");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return hfail(DGSEM_EINVAL, "bad precision");
  for (int d = 0; d < c->nd; ++d)
    if (variants[d] < 0 || variants[d] >= hex::kHexVolVariants)
      return hfail(DGSEM_EINVAL, "domain %d: no element-stiffness variant %d", d, variants[d]);
  for (int d = 0; d < c->nd; ++d) c->vol_variant[precision == DGSEM_FP32_MIXED ? 1 : 0][d] = variants[d];
  return DGSEM_OK;
}

int dghex_autotune(dghex_ctx* c, int precision, int batch, int reps, int* chosen, void* stream) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return hfail(DGSEM_EINVAL, "bad precision");
  if (batch < 1 || reps < 1) return hfail(DGSEM_EINVAL, "batch and reps must be >= 1");
  int rc = ensure_run_state(c, precision, batch);
  if (rc) return rc;
  c->state_valid = false;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == DGSEM_FP32_MIXED ? autotune_impl<float>(c, reps, chosen, s) : autotune_impl<double>(c, reps, chosen, s);
}

int dghex_profile(dghex_ctx* c, int enable) {
  if (!c) return hfail(DGSEM_EINVAL, "ctx is NULL");
  c->profiling = enable != 0;
  for (int k = 0; k < DGHEX_K_COUNT; ++k) {
    c->kernel_ms[k] = 0.0;
    c->launches[k] = 0;
  }
  c->ev_used.clear();
  return DGSEM_OK;
}

int dghex_kernel_stats(const dghex_ctx* c, int kind, double* total_ms, long long* launches) {
  if (!c || kind < 0 || kind >= DGHEX_K_COUNT) return hfail(DGSEM_EINVAL, "bad argument");
  if (total_ms) *total_ms = c->kernel_ms[kind];
  if (launches) *launches = c->launches[kind];
  return DGSEM_OK;
}

void dghex_destroy(dghex_ctx* c) {
  if (!c) return;
  free_run_state(c);
  for (int k = 0; k < 2; ++k) {
    HexDom& D = c->dom[k];
    dfree(D.d_vert); dfree(D.d_elem); dfree(D.d_conn); dfree(D.d_G64); dfree(D.d_G32);
    delete D.basis;
    D.basis = nullptr;
  }
  dfree(c->d_g_fe); dfree(c->d_g_ce); dfree(c->d_g_pt); dfree(c->d_pt_idx); dfree(c->d_g_slot); dfree(c->d_pdat);
  dfree(c->d_g_face);
  dfree(c->d_ftab[0]); dfree(c->d_ftab[1]); dfree(c->d_gtab[0]); dfree(c->d_gtab[1]);
  dfree(c->d_fp_ptr); dfree(c->d_fp_off); dfree(c->d_Bm); dfree(c->d_ent_k); dfree(c->d_modal);
  dfree(c->d_node_ptr); dfree(c->d_node_slot);
  dfree(c->d_Mloc); dfree(c->d_M); dfree(c->d_Minv64); dfree(c->d_Minv32);
  dfree(c->d_step); dfree(c->d_done); dfree(c->d_nf);
  dfree(c->d_damp64); dfree(c->d_damp32); dfree(c->d_rx_gain); dfree(c->d_step_base); dfree(c->d_volt);
  dfree(c->d_zeta64); dfree(c->d_zeta32); dfree(c->d_beta64); dfree(c->d_beta32); dfree(c->d_gamma64);
  dfree(c->d_gamma32);
  for (int k = 0; k < 2; ++k) {
    dfree(c->dom[k].d_pml_elem); dfree(c->dom[k].d_pml_geo64); dfree(c->dom[k].d_pml_geo32);
  }
  dfree(c->d_rw); dfree(c->d_roff); dfree(c->d_rnn);
  dfree(c->d_drive); dfree(c->d_traces);
  for (auto ev : c->ev_pool) cudaEventDestroy(ev);
  delete c;
}

}  // extern "C"
