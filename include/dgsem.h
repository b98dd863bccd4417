/*
 * dgsem.h -- C ABI of the GB300 explicit DG-SEM acoustic step with batched
 * reduced-order PMUT modal coupling (arXiv 2603.06267).
 *
 * The library solves, on one GPU, the semi-discrete system of Sec. 3.1
 *     M p'' + K p = f(q''),      q'' + W q = g(p, phi)        (eqs. semi_SEM, semi_PMUT)
 * where K is the DG-SEM stiffness of eq. (Wf_2): GLL spectral elements, C0
 * inside each box, symmetric interior penalty across the (possibly
 * non-conforming, variable-order) interface Gamma_I between a primary box and
 * a secondary box stacked on its z-max face (Sec. 3, Sec. 5), M the lumped
 * GLL mass, f_i and g_m the membrane integrals of eqs. (f_i) and (g_m), and
 * integrates it with the Newmark gamma = 1/2, beta = 0 predictor/corrector of
 * Algorithm 1.  Walls other than Gamma_PMUT (the primary's z-min face) and
 * Gamma_I are rigid (homogeneous Neumann, eq. full_problem row 7).
 *
 * Conventions common to every call
 *   - Every call returns a dgsem_status; DGSEM_OK is 0, errors are negative.
 *     dgsem_last_error() gives a message for the calling thread's last error.
 *     No call aborts, traps or hangs the GPU; device-side problems are
 *     reported through status words read back by the host.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  Device memory the library allocates belongs to the
 *     context and is released by dgsem_destroy().
 *   - A context is bound to the CUDA device that is current when it is
 *     created; every later call must be made with that device current.
 *   - Node order of full-field vectors (dgsem_set_state, dgsem_get_pressure):
 *     primary lattice then secondary lattice; inside a box, lattice index
 *     (i, j, k) of the GLL nodes with i (x) fastest, i in [0, nelem[0]*order].
 *   - Not thread-safe per context: calls on one context must not overlap.
 */
#ifndef DGSEM_H
#define DGSEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgsem_ctx dgsem_ctx;

typedef enum {
  DGSEM_OK = 0,
  DGSEM_EINVAL = -1,     /* bad argument (null pointer, size, range)            */
  DGSEM_ENOMEM = -2,     /* device or host allocation failed                    */
  DGSEM_ECUDA = -3,      /* a CUDA runtime call failed                          */
  DGSEM_EUNSTABLE = -4,  /* dt above the stability limit, or non-finite state   */
  DGSEM_ETIMEOUT = -5,   /* a bounded device-side wait gave up                  */
  DGSEM_ENOMATCH = -6,   /* interface face matching (Algorithm 3) failed        */
  DGSEM_ESTATE = -7      /* call out of order (e.g. run before pmut_array_set)  */
} dgsem_status;

typedef enum {
  DGSEM_FP64 = 0,        /* every field and operator in FP64                    */
  DGSEM_FP32_MIXED = 1   /* pressure state, volume and face operators in FP32;
                            modal ODEs, membrane projections and receiver traces
                            in FP64                                             */
} dgsem_precision;

/* dgsem_run flags */
#define DGSEM_RUN_CONTINUE 1   /* continue from the context's current state
                                  instead of restarting from rest (p = p' = 0,
                                  q = q' = 0, eq. full_problem row 4, eq. ode
                                  row 3)                                        */

/* One axis-aligned box subdomain meshed by nelem[0] x nelem[1] x nelem[2]
 * equal hexahedra with affine maps X_K (Sec. 3, the affine case of the
 * trilinear maps), GLL order `order` (r_a of V_a^{r_a}, 1 <= order <= 8),
 * sound speed c (m/s) and density rho (kg/m^3). */
typedef struct {
  double origin[3];
  double extent[3];
  int nelem[3];
  int order;
  double c;
  double rho;
} dgsem_domain_desc;

/* Mesh description (Sec. 3 and Sec. 5).
 *   ndomains        1 (primary only) or 2 (primary + secondary).
 *   domains         [ndomains]; domains[0] is the primary box Omega_in, whose
 *                   z-min face carries Gamma_PMUT; domains[1] (if present) is
 *                   Omega_out, stacked on the primary's z-max face with the
 *                   same x-y extent.  Each secondary element face on Gamma_I
 *                   must cover an integer r x r block of primary faces
 *                   (r = 1 conforming, r = 2 the 2:1 case).
 *   fine_faces      NULL, or [n_fine_faces] primary top-layer element columns
 *                   ex + nelem[0]*ey whose z-max face belongs to Gamma_I (the
 *                   "finer" face list of Sec. 5).  NULL = all of them.
 *   coarse_faces    NULL, or [n_coarse_faces] secondary bottom-layer columns
 *                   mx + nelem[0]*my (the "coarser" list).  NULL = all.
 *                   Faces not listed are rigid walls.  The pairs are matched
 *                   by Algorithm 3 (opposite normals, one-vertex radius
 *                   filter, inverse map); a fine-face quadrature node without
 *                   a coarse neighbour fails with DGSEM_ENOMATCH.
 *   dt              time step in s if > 0, else computed from cfl as
 *                   cfl * min_K min_d (h_d/2 * min GLL gap(N_K)) / max c.
 *   penalty_alpha   alpha of gamma_F = alpha cbar^2 max(N)^2 / min(h) (Sec. 3).
 *   iface_quad_pts  Gauss-Legendre points per direction on each fine face;
 *                   0 = max(order) + 1, which integrates the interface terms
 *                   exactly for affine faces. */
typedef struct {
  int ndomains;
  const dgsem_domain_desc* domains;
  int n_fine_faces;
  const int* fine_faces;
  int n_coarse_faces;
  const int* coarse_faces;
  double cfl;
  double dt;
  double penalty_alpha;
  int iface_quad_pts;
} dgsem_mesh_desc;

/* Build the mesh, the 1D GLL/GL tables, the interface maps and the time step
 * on the host and upload them to the current device.  *out receives a new
 * context (NULL on error). */
int dgsem_mesh_create(const dgsem_mesh_desc* desc, dgsem_ctx** out);

/* First-order absorbing boundary (Sec. 2, eq. full_problem row 6, as the
 * damping form d(w, v) = sum_F int_F c w v of eq. Wf_4; matrix C of eq.
 * semi_SEM, diagonal by GLL collocation on the face nodes).
 *   box    0 = primary, 1 = secondary.
 *   sides  [6] for the box sides x-, x+, y-, y+, z-, z+: non-zero = absorbing
 *          (Gamma_ABC), 0 = rigid wall (Gamma_N, the default).  The primary
 *          z-min side (Gamma_PMUT) and the interface sides cannot absorb
 *          (DGSEM_EINVAL).
 * Algorithm 1 applies C to the predicted velocity, explicitly, so dt is held
 * to min(cfl dt, 1 / max_i C_ii/M_ii); a dt the caller fixed in
 * dgsem_mesh_desc above that limit is rejected (DGSEM_EUNSTABLE, nothing
 * changed).  The context's state is invalidated: the next dgsem_run starts
 * from rest. */
int dgsem_set_absorbing(dgsem_ctx* ctx, int box, const int* sides);

/* Perfectly matched layer (Sec. 2, eq. full_problem rows 1-3) inside a box
 * along its sides, with the damping profile of Sec. 2:
 *     zeta_i(x) = zeta~ (s - sin(2 pi s) / (2 pi)),  zeta~ = c / l log(1 / R),
 * s in [0, 1] the depth into a layer of thickness l (0 at its inner face).
 *   box        0 = primary, 1 = secondary.
 *   thickness  [6] layer thickness in m for the sides x-, x+, y-, y+, z-, z+
 *              (0 = none); a layer takes the elements it overlaps.  The
 *              primary z-min side (Gamma_PMUT) and the interface sides
 *              cannot carry one (DGSEM_EINVAL), nor may two layers of an axis
 *              overlap.
 *   R          design reflection coefficient, 0 < R < 1 (the paper uses
 *              1e-5 .. 1e-4).
 * The auxiliary fields Phi (element-local at the GLL nodes of the layer's
 * elements) and psi (nodal) live at half steps like the velocity; Phi's own
 * damping is integrated by Crank-Nicolson, alpha p' acts on the predicted
 * velocity like C p'_pred in Algorithm 1.  dt is held to
 * min(cfl dt, 1 / max_i (C_ii/M_ii + alpha_i)) (the damping terms are
 * explicit); a dt the caller fixed above it is refused (DGSEM_EUNSTABLE).
 * All-zero thickness removes the layer.  The run state is re-allocated and
 * invalidated; checkpoints (dgsem_state_save) of a box with a layer are not
 * supported (DGSEM_ESTATE). */
int dgsem_set_pml(dgsem_ctx* ctx, int box, const double* thickness, double R);

/* Failure-path self test (no counterpart in the paper): one warp waits, with
 * the bounded mbarrier wait the TMA pipeline of the volume kernels uses, on a
 * barrier nothing arrives at; the wait gives up after 2^24 SM clocks and
 * records it in the context's device status word, which this call reads back
 * and clears.  DGSEM_OK when the give-up was reported (a stalled stage in a
 * run is reported the same way, as DGSEM_ETIMEOUT from dgsem_run), DGSEM_ECUDA
 * otherwise.  The context stays usable. */
int dgsem_selftest_wait(dgsem_ctx* ctx, void* stream);

/* Time step, stability bound and size.  dt_stable_max is 2 / sqrt(lambda_max)
 * of M^-1 K from dgsem_check_stability() (0 if it has not run); ndof counts
 * the unique GLL nodes of all boxes (dim V^DG). Any output may be NULL. */
int dgsem_get_dt(const dgsem_ctx* ctx, double* dt, double* dt_stable_max, long long* ndof);

/* Power iteration for lambda_max(M^-1 K) on the device in FP64 (iters
 * products).  Returns DGSEM_EUNSTABLE if dt > 0.95 * 2 / sqrt(lambda_max);
 * *lambda_max (may be NULL) receives the estimate either way. */
int dgsem_check_stability(dgsem_ctx* ctx, int iters, double* lambda_max);

/* GLL nodes of Gamma_PMUT's face lattice (the primary's z-min face):
 * *n_nodes = (nelem[0]*order+1) * (nelem[1]*order+1); *xy points to a
 * library-owned [n_nodes][2] array of (x, y), node index ix + Lx*iy, valid
 * until dgsem_destroy(). */
int dgsem_pmut_nodes(const dgsem_ctx* ctx, int* n_nodes, const double** xy);

/* Reduced-order PMUT array (Sec. 2, eq. pmut_problem; Sec. 3.1 eqs. f_i, g_m).
 *   n_pmut, n_modes  K membranes with M modes each (1 <= M <= 16).
 *   foot_ptr         [K+1] CSR offsets into foot_node / shape_un.
 *   foot_node        [nnz] face-lattice node indices (see dgsem_pmut_nodes)
 *                    of membrane k's footprint gamma_k.
 *   shape_un         [nnz][M] U_{k,m}.n at those nodes (n: outward normal of
 *                    the fluid, -e_z on the z-min face).
 *   freq_hz, damping, eta, modal_mass   [K][M]: omega/2pi, modal damping
 *                    ratio zeta, electromechanical coupling eta (N/V), modal
 *                    mass mu (kg; NULL means 1, the paper's literal ODE).
 * The modal ODE integrated is
 *   mu (q'' + 2 zeta omega q' + omega^2 q) = int_{gamma_k} p U.n dsigma + eta phi,
 * the membrane integrals use GLL collocation on the face nodes, and the
 * acoustic forcing is f_i = -kappa sum q'' int U.n psi_i with kappa = rho c^2
 * of the primary box.  Replaces any previous array; resets the PMUT state. */
int pmut_array_set(dgsem_ctx* ctx, int n_pmut, int n_modes, const int* foot_ptr,
                   const int* foot_node, const double* shape_un, const double* freq_hz,
                   const double* damping, const double* eta, const double* modal_mass);

/* TX -> RX switch of the PMUT array (Sec. 2, eq. ode row 2 / eq.
 * pmut_problem row 2): steps n < n_switch take the drive voltage phi_k,0
 * passed to dgsem_run (transmission); from step n_switch on, membrane k's
 * voltage is the open-circuit value
 *     phi_k^n = sign / C_k * sum_m eta_km q_km^n
 * with the modal coordinates of step n (reception).  n counts steps since
 * the state was at rest or set by dgsem_set_state (dgsem_run flag
 * DGSEM_RUN_CONTINUE keeps counting; checkpoints store the count).
 *   n_switch     first receiving step; < 0 switches reception off (default).
 *   capacitance  [n_pmut] C_k in farads (> 0), copied.
 *   sign         +1: the equation as printed; -1: the convention in which the
 *                open circuit stiffens the membrane (open-circuit frequency
 *                above short-circuit).
 * While reception is configured every dgsem_run records the voltage used in
 * each step, [batch][n_pmut][nsteps] on the device, read with
 * dgsem_get_voltages.  DGSEM_ESTATE without a PMUT array. */
int pmut_set_receive(dgsem_ctx* ctx, long long n_switch, const double* capacitance, int sign);

/* Copy the voltages of the last dgsem_run ([batch][n_pmut][nsteps] doubles,
 * drive before the switch, open circuit after it) to the host array out of n
 * doubles.  DGSEM_ESTATE if that run recorded none, DGSEM_EINVAL if n is too
 * small. */
int dgsem_get_voltages(const dgsem_ctx* ctx, double* out, size_t n);

/* Run nsteps steps of Algorithm 1 for `batch` independent drive patterns
 * sharing the mesh and the PMUT array.
 *   precision  dgsem_precision.
 *   drive      [batch][n_pmut][nsteps] voltages phi_k(t^n), t^n = (n0 + n) dt,
 *              host or device memory (FP64); may be NULL when n_pmut == 0.
 *   recv_xyz   [n_recv][3] receiver positions (host), interpolated with the
 *              tensor Lagrange basis of the containing element (lowest
 *              element id on ties, the primary box on Gamma_I).
 *   traces     [batch][n_recv][nsteps] output (host or device, FP64):
 *              sample n is p^{n0+n+1} at the receivers.
 *   flags      0 or DGSEM_RUN_CONTINUE.
 *   stream     cudaStream_t to order the work on (NULL = legacy default
 *              stream); the call returns after the stream has finished.
 * Without DGSEM_RUN_CONTINUE the state restarts from rest (or from the state
 * given by the last dgsem_set_state/dgsem_state_load) and n0 = 0.
 * Returns DGSEM_EUNSTABLE when the receiver traces or the PMUT state are not
 * finite at the end of the run (the step diverged); the state is then invalid.
 * Any other failure once the run has started (DGSEM_ECUDA, DGSEM_ETIMEOUT,
 * DGSEM_ENOMEM) leaves the state invalid too, so a later DGSEM_RUN_CONTINUE
 * is refused (DGSEM_ESTATE); argument errors found before the run starts
 * leave it as it was. */
int dgsem_run(dgsem_ctx* ctx, int precision, int batch, int nsteps, const double* drive,
              int n_recv, const double* recv_xyz, double* traces, int flags, void* stream);

/* Several meshes in one launch: dgsem_run on each of the n contexts with the
 * same precision, nsteps and flags, their time steps captured as parallel
 * branches of one CUDA graph so that meshes of different sizes and orders
 * (e.g. PMUT arrays of different sizes) share the GPU in one launch.  All
 * contexts must belong to the current device and be distinct.  Per-context
 * arrays: batch[n], drive[n] (as in dgsem_run), n_recv[n], recv_xyz[n],
 * traces[n]; n_recv, recv_xyz and traces may be NULL when no context has
 * receivers.  Results equal n separate dgsem_run calls. */
int dgsem_run_multi(int n, dgsem_ctx* const* ctxs, int precision, const int* batch, int nsteps,
                    const double* const* drive, const int* n_recv, const double* const* recv_xyz,
                    double* const* traces, int flags, void* stream);

/* Initial state p^0, p'^0 (host, FP64, [ndof] in the node order above,
 * broadcast to every batch member) for the next dgsem_run without
 * DGSEM_RUN_CONTINUE; the run starts from p''^0 = M^-1 (-K p^0).  Either
 * pointer may be NULL (zero). */
int dgsem_set_state(dgsem_ctx* ctx, const double* p0, const double* v0);

/* Leapfrog energy of the acoustic field of every batch member after the
 * last run (diagnostics, computed in FP64 for either state precision): e[b]
 * = 1/2 v^T M v + 1/2 p^n^T K p^{n+1} with v = v^{n+1/2} and K the stiffness
 * with the interface terms (no PMUT coupling, absorbing or layer terms);
 * Algorithm 1 conserves it exactly without forcing and damping.  An FP32
 * state is widened to FP64 copies first (about three state-sized FP64
 * buffers per box, allocated for the call; DGSEM_ENOMEM if they do not fit).
 * e holds n >= batch values. */
int dgsem_energy(dgsem_ctx* ctx, double* e, int n);

/* Modal state of the PMUT array after the last run: q^n, q'^n, q''^n of
 * every batch member, PMUT and mode, each a host array [batch][n_pmut]
 * [n_modes] of n >= batch * n_pmut * n_modes doubles (any pointer may be
 * NULL).  DGSEM_ESTATE without a PMUT array or a state. */
int dgsem_get_pmut_state(const dgsem_ctx* ctx, double* q, double* qd, double* qdd, size_t n);

/* Current pressure field p^n of every batch member after the last run, as
 * FP64 host array [batch][ndof] (node order above). */
int dgsem_get_pressure(const dgsem_ctx* ctx, double* p, size_t len);

/* Checkpoint of the full time-stepping state (pressure pair, half-step
 * velocity, PMUT q, q', q'', step counter, precision, batch).  With buf NULL,
 * *len receives the size needed; otherwise *len must hold the buffer size. */
int dgsem_state_save(const dgsem_ctx* ctx, void* buf, size_t* len);
int dgsem_state_load(dgsem_ctx* ctx, const void* buf, size_t len);

/* Tile shapes of the fused volume kernel.  Orders 4 and 6 have several
 * CTA tile shapes (element columns x element rows); dgsem_num_tiles gives
 * their count for a box and precision, dgsem_set_tiles selects one per box
 * ([ndomains] variant indices, 0 = default) for later runs at that
 * precision, and dgsem_autotune times every variant of each box's volume
 * kernel for `batch` patterns (`reps` launches each, CUDA events on `stream`)
 * and keeps the fastest (written to chosen[ndomains] if not NULL).  The
 * autotuner uses the run state as scratch: the next dgsem_run must not pass
 * DGSEM_RUN_CONTINUE. */
int dgsem_num_tiles(const dgsem_ctx* ctx, int precision, int box, int* n);
int dgsem_set_tiles(dgsem_ctx* ctx, int precision, const int* tiles);
int dgsem_autotune(dgsem_ctx* ctx, int precision, int batch, int reps, int* chosen, void* stream);

/* Launch shape of the fused volume kernels (no counterpart in the paper).
 * A CTA owns an x-y tile of a box and marches through a chunk of its
 * element layers in z, streaming one layer after another through a ring of
 * shared-memory stages.  dgsem_set_layers sets, per box, the layers one CTA
 * marches through ([ndomains] values; 0 = automatic, the default: all of the
 * box's layers, halved while the grid would have fewer than 4 x 152 CTAs;
 * values above the box's layer count are clamped to it).  The value applies to
 * every later launch at either precision.  dgsem_vol_launch reports the shape
 * of box `box`'s volume launch in the last dgsem_run: shape[8] = grid x, y, z,
 * block x, y, z, layers per CTA, z chunks (grid z = z chunks x batch).
 * DGSEM_ESTATE before the first run. */
int dgsem_set_layers(dgsem_ctx* ctx, const int* layers_per_cta);
int dgsem_vol_launch(const dgsem_ctx* ctx, int box, int* shape);

/* Kernel instrumentation.  dgsem_profile(ctx, 1) makes later runs bracket
 * every kernel launch with CUDA events on the run's stream; statistics are
 * accumulated per kernel kind (DGSEM_K_*) until dgsem_profile(ctx, 1) is
 * called again (which resets them) or profiling is switched off with 0.
 * Launch counts are kept whether or not timing is enabled. */
#define DGSEM_K_PMUT_RECV 0   /* PMUT modal step + receiver sampling          */
#define DGSEM_K_IFACE 1       /* interface fluxes on Gamma_I                   */
#define DGSEM_K_VOL0 2        /* fused volume update of the primary box        */
#define DGSEM_K_VOL1 3        /* fused volume update of the secondary box      */
#define DGSEM_K_PML 4         /* perfectly matched layer elements (both boxes) */
#define DGSEM_K_COUNT 5
int dgsem_profile(dgsem_ctx* ctx, int enable);
int dgsem_kernel_stats(const dgsem_ctx* ctx, int kind, double* total_ms, long long* launches);

/* Receiver sampling that allocates no device memory (the paper has no
 * counterpart; this is a service of this library).
 *
 * Samples the current pressure field p^n of every batch member (the state
 * left by the last dgsem_run) at n_recv points, with the same element choice
 * and tensor Lagrange interpolation as dgsem_run's traces.
 *   recv_xyz  [n_recv][3] positions, host or device memory.
 *   out       [batch][n_recv] FP64, device memory (written on `stream`).
 *   out_len   number of doubles `out` holds; less than batch * n_recv is
 *             refused (DGSEM_EINVAL) before anything is written.
 * Why: some callers cannot call cudaMalloc when they want a sample -- a
 * process whose device memory has been handed out entirely to another
 * allocator (for instance a framework's caching pool that reserved the GPU),
 * or code running under a fixed device-memory budget that a new buffer would
 * exceed.  This call allocates nothing: its receiver table lives in one
 * fixed array of about 0.75 MiB that every device loading the library holds
 * until the process exits.
 * Limits and behaviour:
 *   - at most 64 receivers per call (larger n_recv returns DGSEM_EINVAL with
 *     a message); a receiver outside the mesh returns DGSEM_EINVAL and leaves
 *     the context usable; needs a previous dgsem_run (DGSEM_ESTATE otherwise).
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it; make that first call before any
 *     stream capture begins.  The kept address is not refreshed after
 *     cudaDeviceReset.
 *   - the call reads a status word back and waits for `stream` (it returns
 *     after the stream has finished the work).
 *   - all calls share the one array and it keeps the last call's contents
 *     (the status word is cleared at every call, the table is overwritten),
 *     so calls whose work overlaps on the GPU (other host threads, other
 *     streams) race: issue them one at a time. */
int dgsem_sample_noalloc(dgsem_ctx* ctx, int n_recv, const double* recv_xyz, double* out, size_t out_len,
                         void* stream);

/* Arithmetic-rate probe (no counterpart in the paper; measurement support).
 * Runs long chains of independent fused multiply-adds on every SM of the
 * current device -- plain FP64 DFMA for DGSEM_FP64, packed f32x2 FMA for
 * DGSEM_FP32_MIXED -- in launches of about 0.2 s timed with CUDA events on
 * `stream`, and writes the best of three rates in TFLOP/s (2 flops per FMA)
 * to *tflops.  It reads the clocks the GPU runs at and changes no setting.
 * Allocates a small output buffer for the call. */
int dgsem_measure_peak(int precision, double* tflops, void* stream);

/* Message of the calling thread's last error ("" if none). */
const char* dgsem_last_error(void);

/* Release every device and host resource of the context (NULL is a no-op). */
void dgsem_destroy(dgsem_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DGSEM_H */
