/*
 * dghex.h -- C ABI of the explicit DG-SEM acoustic step on general
 * hexahedral meshes (trilinear elements) with batched reduced-order PMUT
 * coupling (arXiv 2603.06267).
 *
 * Same method as dgsem.h (semi-discrete system of Sec. 3.1, eqs. semi_SEM /
 * semi_PMUT, integrated with Algorithm 1), on meshes whose elements are
 * K = X_K(K^) with a trilinear invertible map X_K of positive Jacobian
 * (Sec. 3) instead of equal axis-aligned boxes:
 *   - the volume term of eq. (Wf_2) uses per-node geometric factors
 *     c^2 w_abc |J| J^-1 J^-T at the element's GLL nodes;
 *   - the interface Gamma_I between the fine primary domain and the coarse
 *     secondary domain is given by two face lists and matched on the GPU by
 *     Algorithm 3 (normal filter, one stored vertex per coarse face within
 *     r = max(diam) + eps of the fine quadrature node, Newton-Raphson for the
 *     reference position, containment in [-1, 1]^3); its SIPG terms are
 *     integrated on Gauss-Legendre nodes of the fine faces (Sec. 5) with the
 *     surface Jacobian |J| |J^-T e| (Nanson) and the normal at each node;
 *   - Gamma_PMUT is a list of primary boundary faces.
 * Readings where the paper is silent (documented with the oracle as well):
 * the matching filter uses each face's normal at its centre; h of gamma_F is
 * |K| / |F| (GLL rule of the element's order), minimum over the two sides at
 * each quadrature node; the CFL length of an element is its shortest edge;
 * a receiver lies in the lowest-id element (primary first) whose Newton
 * reference position is within [-1, 1]^3 up to 1e-10.
 *
 * Status codes, precisions, dgsem_last_error() and the ownership rules are
 * those of dgsem.h.  All other boundary faces are rigid walls.
 *
 * Element convention: an element lists 8 vertex ids; corner (i, j, k) in
 * {0, 1}^3 is at list position i + 2 j + 4 k and is the image of reference
 * corner (2i-1, 2j-1, 2k-1).  Local face f = 2 * axis + side is the face
 * xi_axis = -1 (side 0) or +1 (side 1).  Elements may be listed in any
 * orientation; the C0 node numbering matches shared vertices, edges and
 * faces topologically.
 *
 * Node order of full-field vectors: every node of domain 0 then every node
 * of domain 1; inside a domain, the nodes of each mesh entity (vertex, edge,
 * face, element interior) get consecutive numbers when the entity first
 * appears, scanning the elements in order and each element's nodes by local
 * GLL index a + (N+1) b + (N+1)^2 c.  dghex_nodes gives their positions.
 */
#ifndef DGHEX_H
#define DGHEX_H

#include <stddef.h>
#include "dgsem.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dghex_ctx dghex_ctx;

/* One domain: GLL order (1..8), sound speed c (m/s), density rho (kg/m^3),
 * vertices [n_vert][3] (m) and elements [n_elem][8] vertex ids (convention
 * above).  Every element must have a positive Jacobian at its GLL nodes. */
typedef struct {
  int order;
  double c;
  double rho;
  int n_vert;
  const double* vert;
  int n_elem;
  const int* elem;
} dghex_domain_desc;

/* Mesh description.
 *   ndomains         1 or 2; domains[0] is the fine primary (carries
 *                    Gamma_PMUT), domains[1] the coarse secondary.
 *   fine_faces       [n_fine_faces][2] (element, local face) of domain 0 on
 *                    Gamma_I; coarse_faces [n_coarse_faces][2] of domain 1.
 *                    Needed when ndomains == 2, ignored otherwise.
 *   pmut_faces       [n_pmut_faces][2] (element, local face) of domain 0 on
 *                    Gamma_PMUT (may be 0 / NULL).
 *   cfl              dt = cfl * min_K (h_min,K / 2 * min GLL gap(N_K)) / max c
 *                    when dt <= 0.
 *   dt               fixed time step (s), or <= 0 to use cfl.
 *   penalty_alpha    alpha of gamma_F = alpha cbar^2 max(N)^2 / h (> 0).
 *   iface_quad_pts   Gauss points per direction on each fine face (0: the
 *                    larger order + 1; at most 9).
 *   normal_tol       Algorithm 3 filter |n+ + n-| < normal_tol (0: 0.5).
 * Errors: DGSEM_EINVAL for bad sizes, ids, faces that are not boundary faces,
 * or a non-positive Jacobian; DGSEM_ENOMATCH if a fine quadrature node has
 * no coarse neighbour. */
typedef struct {
  int ndomains;
  const dghex_domain_desc* domains;
  int n_fine_faces;
  const int* fine_faces;
  int n_coarse_faces;
  const int* coarse_faces;
  int n_pmut_faces;
  const int* pmut_faces;
  double cfl;
  double dt;
  double penalty_alpha;
  int iface_quad_pts;
  double normal_tol;
} dghex_mesh_desc;

int dghex_mesh_create(const dghex_mesh_desc* desc, dghex_ctx** out);

/* Time step and the number of unique GLL nodes of all domains (dim V^DG).
 * Either output may be NULL. */
int dghex_get_dt(const dghex_ctx* ctx, double* dt, long long* ndof);

/* Positions of all nodes, [ndof][3] library-owned (valid until destroy), and
 * the first node of domain 1 (= ndof with one domain). */
int dghex_nodes(const dghex_ctx* ctx, long long* ndof, long long* first_secondary, const double** xyz);

/* Nodes of Gamma_PMUT: *n unique nodes on the PMUT faces (ascending node
 * id), positions [n][3] and assembled face weights W_j = sum_F w_a w_b |J_F|
 * [n] (library-owned).  pmut_nodes[j] is an index into this list. */
int dghex_pmut_nodes(const dghex_ctx* ctx, int* n, const double** xyz, const double** weight);

/* Reduced-order PMUT array on Gamma_PMUT (eq. pmut_problem; eqs. f_i, g_m).
 * Arguments as pmut_array_set in dgsem.h, with foot_node indices into the
 * dghex_pmut_nodes list and shape_un = U_{k,m}.n at those nodes (n the
 * outward normal of the fluid). B_{j,km} = W_j U_{k,m}(x_j).n, kappa =
 * rho c^2 of domain 0.  Resets the PMUT state. */
int dghex_pmut_set(dghex_ctx* ctx, int n_pmut, int n_modes, const int* foot_ptr, const int* foot_node,
                   const double* shape_un, const double* freq_hz, const double* damping, const double* eta,
                   const double* modal_mass);

/* First-order absorbing faces (Gamma_ABC) of one domain (eq. Wf_4): the
 * damping form d(w, v) = sum_F int_F c w v, collocated at the faces' GLL
 * nodes with the Nanson surface Jacobian (C diagonal), acting on the
 * predicted velocity as in Algorithm 1.  faces [n][2] (element, local face)
 * must be boundary faces of that domain and not on Gamma_I or Gamma_PMUT;
 * n = 0 removes the domain's absorbing faces.  dt is held to
 * min(cfl dt, 1 / max_j C_jj / M_jj); a dt fixed at creation above that
 * bound is refused (DGSEM_EUNSTABLE).  The state restarts from rest. */
int dghex_set_absorbing_faces(dghex_ctx* ctx, int domain, int n, const int* faces);

/* Perfectly matched layers (Sec. 2, eq. full_problem rows 1-3) along the
 * sides x-, x+, y-, y+, z-, z+ of a domain's bounding box, thickness[6] in m
 * (0 = none), design reflection R in (0, 1) (one R per mesh), with the
 * profile zeta~ (s - sin(2 pi s) / (2 pi)), zeta~ = c / l log(1/R), s the
 * depth into the layer.  As on the box path (dgsem_set_pml): psi nodal, Phi
 * element-local at the GLL nodes of the layer elements (any node with a
 * non-zero profile), gradients J^-T grad^ on the curved elements,
 * Crank-Nicolson damping of Phi, alpha p' on the predicted velocity; dt held
 * to 1 / max (C/M + alpha).  All-zero thickness removes the domain's layers.
 * The state restarts from rest; checkpoints of a state with a layer are
 * refused (DGSEM_ESTATE). */
int dghex_set_pml(dghex_ctx* ctx, int domain, const double* thickness, double R);

/* TX -> RX switch and the voltage record, as pmut_set_receive and
 * dgsem_get_voltages in dgsem.h (steps counted since rest or the last
 * dghex_set_state; DGSEM_RUN_CONTINUE and checkpoints keep counting). */
int dghex_pmut_set_receive(dghex_ctx* ctx, long long n_switch, const double* capacitance, int sign);
int dghex_get_voltages(const dghex_ctx* ctx, double* out, size_t n);

/* Checkpoint of the time-stepping state (pressure, half-step velocity,
 * PMUT forcing rows, q, q', q'', step count, precision, batch), as
 * dgsem_state_save / dgsem_state_load.  A loaded state is continued by the
 * next dghex_run with DGSEM_RUN_CONTINUE. */
int dghex_state_save(const dghex_ctx* ctx, void* buf, size_t* len);
int dghex_state_load(dghex_ctx* ctx, const void* buf, size_t len);

/* Algorithm 3 result: for every fine face (list order) and every Gauss node
 * (s fastest, s and t the face's two other reference axes in increasing
 * order), the index of the matched coarse face in coarse_faces and the
 * reference position in its element.  coarse_face [n_fine_faces * q * q],
 * ref [n_fine_faces * q * q][3]; *q receives q.  Either array may be NULL;
 * n is the number of points the arrays hold. */
int dghex_get_matches(const dghex_ctx* ctx, int* q, int* coarse_face, double* ref, long long n);

/* Run nsteps steps of Algorithm 1 for `batch` drive patterns (arguments,
 * flags, trace convention, the DGSEM_EUNSTABLE divergence report and the
 * invalid state after a failed run as dgsem_run in dgsem.h). */
int dghex_run(dghex_ctx* ctx, int precision, int batch, int nsteps, const double* drive, int n_recv,
              const double* recv_xyz, double* traces, int flags, void* stream);

/* Initial state p^0, p'^0 ([ndof] FP64 host, node order above; NULL = 0)
 * for the next run without DGSEM_RUN_CONTINUE: p''^0 = M^-1 (-K p^0 - C p'^0)
 * (C: absorbing faces). */
int dghex_set_state(dghex_ctx* ctx, const double* p0, const double* v0);

/* Leapfrog energy of the acoustic field of every batch member after the
 * last run (FP64 state only; diagnostics): e[b] = 1/2 v^T M v + 1/2 p^n^T K
 * p^{n+1} with v = v^{n+1/2}, K the stiffness with the interface terms (no
 * PMUT coupling, absorbing or layer terms).  Algorithm 1 conserves it
 * exactly without forcing and damping.  e holds n >= batch values. */
int dghex_energy(dghex_ctx* ctx, double* e, int n);

/* Pressure p^n of every batch member after the last run, [batch][ndof]. */
int dghex_get_pressure(const dghex_ctx* ctx, double* p, size_t len);

/* Power iteration for lambda_max(M^-1 K) on the device in FP64 (iters
 * products, with the step's own stiffness and interface kernels, from a fixed
 * pseudo-random start vector).  Returns DGSEM_EUNSTABLE if dt > 0.95 * 2 /
 * sqrt(lambda_max) (the explicit scheme's limit; the CFL rule of
 * dghex_mesh_create is a heuristic on distorted elements); *lambda_max (may
 * be NULL) receives the estimate either way.  Uses the run state as scratch:
 * the next dghex_run starts afresh. */
int dghex_check_stability(dghex_ctx* ctx, int iters, double* lambda_max);

/* Interface kernel.  When every Gauss node of a (fine face, coarse element)
 * group lies on one face of each side's element (a geometrically conforming
 * interface; checked at mesh creation to 1e-12 in the coarse reference
 * coordinate), the interface terms are evaluated on collapsed face arrays;
 * otherwise by full tensor evaluation at each node.  general = 1 forces the
 * full evaluation (0 restores the automatic choice).  Both give the same
 * operator up to rounding. */
int dghex_set_interface_kernel(dghex_ctx* ctx, int general);

/* Launch variants of the element-stiffness kernel of eq. (Wf_2).  They do the
 * same arithmetic in the same order (results agree bit for bit) and differ in
 * batch members per thread, elements per CTA and what is kept in registers,
 * shared memory or the read-only cache, i.e. in resident CTAs per SM.  They
 * differ only for batches of at least the vector width (8 FP32, 4 FP64
 * members) and orders >= 3; elsewhere every index runs the default kernel.
 * dghex_num_volume_variants writes their count; dghex_set_volume_variant
 * selects one per domain (variants[ndomains], 0 = default) for later runs at
 * `precision`; dghex_autotune times every variant of each domain's kernel for
 * `batch` patterns (one warm-up and `reps` timed launches, CUDA events on
 * `stream`), keeps the fastest and writes it to chosen[ndomains] (may be
 * NULL).  The autotuner uses the run state as scratch: the next dghex_run
 * must not pass DGSEM_RUN_CONTINUE.  DGSEM_EINVAL for an index out of range,
 * batch < 1 or reps < 1. */
int dghex_num_volume_variants(const dghex_ctx* ctx, int* n);
int dghex_set_volume_variant(dghex_ctx* ctx, int precision, const int* variants);
int dghex_autotune(dghex_ctx* ctx, int precision, int batch, int reps, int* chosen, void* stream);

/* Kernel instrumentation as dgsem_profile / dgsem_kernel_stats. */
#define DGHEX_K_PMUT 0       /* PMUT modal step                                   */
#define DGHEX_K_VOL 1        /* element stiffness (both domains)                  */
#define DGHEX_K_IFACE 2      /* interface fluxes                                  */
#define DGHEX_K_UPDATE 3     /* assembly of the element residuals + leapfrog update */
#define DGHEX_K_TAIL 4       /* PMUT forcing rows + receiver sampling             */
#define DGHEX_K_PML 5        /* perfectly matched layer elements                  */
#define DGHEX_K_COUNT 6
int dghex_profile(dghex_ctx* ctx, int enable);
int dghex_kernel_stats(const dghex_ctx* ctx, int kind, double* total_ms, long long* launches);

/* Release the context (NULL is a no-op). */
void dghex_destroy(dghex_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DGHEX_H */
