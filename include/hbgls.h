/*
 * hbgls.h -- C ABI of the GB300 harmonic balance (HB) Galerkin/least-squares Navier-Stokes library.
 *
 * The library evaluates and solves the discrete HB-GLS equations of arXiv 2411.14315 (Sec. 2):
 * incompressible Newtonian flow on P1 tetrahedra with equal-order velocity and pressure, the solution
 * represented by its values at N = 2 n_h + 1 equally spaced instances of one period T (Eq. upghharm),
 * coupled in time by H = E^-1 Omega E (Eq. NS-harm), stabilised by GLS with the per-instance tau of
 * Eq. (tau), and solved by pseudo-time-stepped Newton-Krylov iterations (Eqs. NR, splitK; Sec. 2.3).
 *
 * Conventions (every entry point):
 *  - Every function returns an hb_status; HB_OK is 0.  Nothing throws across the ABI.  On failure,
 *    hb_last_error() returns a thread-local message describing the last error of this thread.
 *  - The caller owns every array it passes.  Host arrays are read (or written) during the call only
 *    and are never retained; the library copies what it keeps.  `_dev` entry points take device
 *    pointers owned by the caller, valid for the duration of the work queued on the given stream.
 *  - Instance layout ("instances"): double (or float) [n_nodes][4][N], fields u1, u2, u3, p, the N
 *    instances t_n = n T / N contiguous.  Harmonic layout ("harmonics"): double
 *    [n_nodes][4][2 n_h + 1], per field (a0, a1, b1, ..., a_nh, b_nh) of the real series
 *    f(t) = a0 + sum_k a_k cos(k w t) + b_k sin(k w t), w = 2 pi / T.
 *  - Waveform arguments `a`, `b` have n_h + 1 entries (b[0] ignored) in the same real series; they are
 *    the truncated Fourier data of a boundary condition (Eq. upgh_def).
 *  - Units are the caller's (the paper uses cgs).
 *  - A problem is bound to one device and one stream; calls on one problem must not overlap in time
 *    from several host threads.
 */
#ifndef HBGLS_H
#define HBGLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HB_OK = 0,
    HB_ERR_INVALID_ARG = 1,   /* null pointer, size or tag out of range */
    HB_ERR_MESH = 2,          /* degenerate tetrahedron, face not on the mesh, index out of range */
    HB_ERR_CUDA = 3,          /* a CUDA runtime call failed (message carries the CUDA error string) */
    HB_ERR_OOM = 4,           /* device allocation failed */
    HB_ERR_NOT_CONVERGED = 5, /* solve stopped at its iteration limit; best state kept */
    HB_ERR_NAN = 6,           /* residual became NaN/Inf; last finite state kept */
    HB_ERR_TIMEOUT = 7,       /* a bounded device wait of the pipelined element pass gave up (reported by
                                 the next call that synchronises: a host-buffer entry point or hb_solve) */
    HB_ERR_STATE = 8          /* call out of order (e.g. solve before any inflow is set) */
} hb_status;

typedef struct hb_problem hb_problem;    /* opaque; owned by the library, freed by hb_destroy */

/* Mesh of linear tetrahedra (Sec. 2.3, P1 interpolation).  Boundary triangles carry a tag: tag 0 is a
 * no-slip wall (u = 0, stationary walls as in Sec. 2.1); positive tags are caps whose condition is set
 * by hb_set_inflow / hb_set_outlet_*; a cap with no condition is traction free (h = 0).
 * The local vertex order of each tetrahedron is significant: tau's metric is that of the map to the
 * parent tetrahedron with local vertex 0 at its origin (Eq. tau). */
typedef struct {
    int64_t n_nodes, n_tets, n_faces;
    const double *xyz;        /* [n_nodes][3] */
    const int32_t *tets;      /* [n_tets][4], 0-based node ids */
    const int32_t *faces;     /* [n_faces][3] boundary triangles, any orientation */
    const int32_t *face_tag;  /* [n_faces] */
} hb_mesh;

/* Create a problem (Eq. NS-time data): density rho > 0, dynamic viscosity mu > 0, period T > 0 and
 * n_h >= 0 retained harmonics, N = 2 n_h + 1 <= 31 instances.  Builds the element patches, geometry
 * and boundary data on `device`; `cuda_stream` (a cudaStream_t, may be NULL for a library-owned
 * stream) orders all later device work of this problem.  Errors: INVALID_ARG, MESH, CUDA, OOM. */
hb_status hb_create(const hb_mesh *mesh, double rho, double mu, double period_T, int n_h, int device,
                    void *cuda_stream, hb_problem **out);
/* Free a problem and all its device memory; NULL is accepted (HB_OK). */
hb_status hb_destroy(hb_problem *p);
/* Message of the last failed call on this thread (thread-local; later successful calls keep it). */
const char *hb_last_error(void);

/* Dirichlet inflow on cap `tag` (Eq. NS-time, u = g on Gamma_g): g(x, t) = profile(x) q(t) with
 * q the waveform (a, b).  profile: [n_nodes][3] (read at the cap's nodes only), or NULL for the
 * parabolic profile at unit flow rate: (2 / (pi R^2)) max(0, 1 - r^2 / R^2) along the inward normal,
 * R the largest in-plane distance of a cap node from the cap's area-weighted centroid.  Nodes shared
 * with a wall keep u = 0; nodes shared by two inflow caps take the values of the cap set last (a
 * repeated call for the same tag replaces it in place).  Errors: INVALID_ARG (tag 0 or unknown). */
hb_status hb_set_inflow(hb_problem *p, int tag, const double *profile, const double *a, const double *b);
/* Dirichlet inflow on cap `tag` from general per-point data (Eq. upgh_def gives Fourier coefficients
 * g*_m(x) per point): harmonics [n_nodes][3][2 n_h + 1] in the real layout (a0, a1, b1, ...), read at
 * the cap's nodes.  Same precedence rules as hb_set_inflow. */
hb_status hb_set_inflow_harmonics(hb_problem *p, int tag, const double *harmonics);
/* Outlet at fixed pressure P(t) (Sec. 3 uses steady values): traction h = -P on cap `tag`. */
hb_status hb_set_outlet_pressure(hb_problem *p, int tag, const double *a, const double *b);
/* Resistance outlet -- an extension the paper leaves out of scope (Sec. 3 and Sec. 4):
 * h_n = -(P_d(t_n) + R Q_n), Q_n the outflow rate through the cap at instance n. */
hb_status hb_set_outlet_resistance(hb_problem *p, int tag, double R, const double *a, const double *b);
/* Backflow stabilisation coefficient beta in [0, 1] on every Neumann face (Sec. 2.3; default 0.2). */
hb_status hb_set_backflow(hb_problem *p, double beta);

/* Stabilisation variants of Sec. 2.2 (the remarks after Eq. tau).  variant 0: the GLS form of Eq. (NS-weak)
 * as printed (default); variant 1: full RBVMS -- the subscale velocity u' = -tau L / rho is also added to
 * the advecting velocity of the Galerkin convective term, which adds the cross stress
 * int N_A rho u' . grad u_i and the Reynolds stress -int rho (u' . grad N_A) u'_i to the momentum rows of
 * the residual and of the exact Jacobian (the paper's tangent keeps its GLS blocks).  ct_dt >= 0 adds
 * ct_dt (1 / dt)^2 under the root of Eq. (tau) with the equivalent step dt = 2 pi / (N w) = T / N (0: Eq.
 * tau as printed; 1: the remark's (1/dt)^2).  Applies to every later evaluation and solve of the problem
 * (not to hb_march, which uses tau_hat of Eq. tauhat).  Synchronises the problem's stream; drops the last
 * assembly of hb_assemble_dev.  Errors: INVALID_ARG for another variant or a negative / non-finite ct_dt. */
hb_status hb_set_stabilization(hb_problem *p, int variant, double ct_dt);

/* Element-to-node summation of every later evaluation (residual, Jv of kinds 0-2, Jacobi diagonal,
 * assembly) and solve of the problem.  The element integrals of Eq. (Rmc) and of the tangent blocks
 * (Eqs. K_mat, ctangent, F_mat) are summed into each node's rows:
 *   1 (default): with floating-point atomics from the element and face kernels; the order of the
 *      additions, and so the last bits of the result, can change from run to run;
 *   0: deterministic.  Each element stores its contributions in its own slot
 *      ([element][4 nodes][4 or 7 fields][N]) and each Neumann face in its own
 *      ([face][3 nodes][3 fields][N]); one gather kernel per call sums every node's slots in a fixed
 *      order (elements in patch order, then faces), and the row-wise assembly adds a node's element
 *      blocks in element order.  Resistance-outlet flow rates are summed in face order by one block per
 *      outlet and instance.  No floating-point atomics run, so equal inputs give bitwise equal outputs.
 *      Device memory: about 64 N (FP32) or 128 N (FP64) bytes per element for the paper tangent, 112 N
 *      or 224 N for the residual and the exact Jacobian, allocated on first use.
 * hb_jv_dev_noalloc and batch layouts 0 and 1 keep the atomic summation (hb_batch_set_grouping).
 * Synchronises the problem's stream; drops the last assembly.  INVALID_ARG for another value;
 * hb_get_scatter returns the current setting (-1 for a null problem). */
hb_status hb_set_scatter(hb_problem *p, int scatter);
int hb_get_scatter(const hb_problem *p);

/* Initial state from harmonics ([n_nodes][4][2 n_h + 1]) or NULL for the default: Dirichlet values
 * built in (Sec. 2.3), zero interior velocity, pressure at the mean outlet level.  Dirichlet values
 * always overwrite the velocity of Dirichlet nodes. */
hb_status hb_set_initial(hb_problem *p, const double *harmonics);
/* Same, from instance values [n_nodes][4][N]. */
hb_status hb_set_instances(hb_problem *p, const double *instances);

typedef struct {
    int precision;            /* 0: every kernel FP64 ("plain FP64"); 1: mixed -- FP32 Jv, FP64 residual,
                                 Arnoldi, norms and update */
    double rtol;              /* stop when ||r|| <= rtol ||r0|| and ||dy|| <= 10 rtol ||y||            */
    double switch_rtol;       /* pseudo-time phase (paper tangent) until ||r|| / ||r0|| < switch_rtol
                                 (Sec. 2.3 uses 1e-3 as its whole convergence criterion); then exact
                                 Newton                                                               */
    double gmres_rtol_pseudo; /* GMRES tolerance in the pseudo phase (paper: 0.03)                     */
    double gmres_rtol_newton; /* GMRES tolerance in the Newton phase                                   */
    int gmres_restart;        /* Krylov basis size m (<= 200)                                          */
    int max_gmres;            /* GMRES iteration cap per linear solve                                  */
    int max_steps;            /* outer (pseudo + Newton) step cap                                      */
    double dt_pseudo;         /* pseudo time step; <= 0 selects the CFL rule of Sec. 2.3               */
    double cfl;               /* CFL number of that rule (1)                                           */
    int use_learned;          /* with a network attached (not the paper's method): 1 = start from its
                                 prediction (warm start); 2 = learned correction step: start from the
                                 current state and, before each linear solve, take the least-squares
                                 multiple of (prediction - state) against its Jacobian image, then plain
                                 GMRES on the remaining residual (the fallback when the prediction does
                                 not help); HB_ERR_INVALID_ARG for other values                          */
    int verbose;              /* print one line per outer step to stderr                               */
    int ser;                  /* 1: switched evolution relaxation -- the pseudo step grows as
                                 ||r0|| / ||r|| (an extension; the paper keeps dt fixed; the converged
                                 state is the same root)                                              */
    double ser_max;           /* cap of that growth factor                                             */
    double r_ref;             /* > 0: residual scale of rtol and switch_rtol instead of ||r0|| (lets a
                                 warm-started solve stop at the same absolute residual as a cold one)  */
    int assembled;            /* 1: in the paper-tangent phase assemble the tangent once per step
                                 (hb_assemble_dev) and let GMRES apply it as a sparse product          */
    int precond;              /* 0: Jacobi on diag(P) + shift M (Sec. 2.3); 1: node blocks (4 x 4 per
                                 node and instance) of the assembled paper tangent + shift M, inverted
                                 through their pressure Schur complement; 2: one V-cycle of aggregation
                                 multigrid on the assembled paper tangent + shift M (greedy node
                                 aggregates, Galerkin coarse operators, damped node-block Jacobi
                                 smoothing; after two consecutive linear solves that stop at max_gmres
                                 with more than half of their right-hand side left the solve
                                 continues with 0); 1 and 2 are
                                 extensions that assemble the tangent every outer step                 */
    int line_search;          /* 1 (default): after the switch, exact Newton without the pseudo shift and a
                                 backtracking line search on ||r|| (step halved up to 4 times until
                                 ||r|| falls by at least 1e-4 of the step fraction; if none does, the
                                 step is retaken with the pseudo shift); 0: the pseudo shift stays in the
                                 Newton phase until dt exceeds ser_max times the CFL step (an extension
                                 either way; the paper stops at the switch criterion, Sec. 2.3)        */
    int scatter;              /* element-to-node summation (Sec. 2.2's assembly of the element
                                 integrals): 1 (default) floating-point atomics; 0 deterministic (the
                                 colour-free equivalent of a colour-class scatter, see hb_set_scatter).
                                 hb_solve applies it to the problem (it stays set afterwards)          */
    double backflow_beta;     /* >= 0: backflow stabilisation coefficient beta in [0, 1] (Sec. 2.3),
                                 applied to the problem as hb_set_backflow would (it stays set); < 0
                                 (default): keep the problem's value                                   */
} hb_solve_opts;

typedef struct {
    int steps, newton_steps, gmres_iters, jv_calls, residual_calls;
    double res0, res_final, seconds, dt_pseudo;
    int status;               /* hb_status of the solve */
} hb_report;

/* Fill the defaults of every field (the paper's settings of Sec. 2.3 where it states them: GMRES
 * tolerance 0.03 in the pseudo-time phase, switch to Newton at ||r|| / ||r0|| < 1e-3).  INVALID_ARG for
 * NULL. */
hb_status hb_default_opts(hb_solve_opts *o);
/* Solve for the periodic state (Eq. NR with the split tangent of Eq. splitK and pseudo time stepping).
 * The state of the problem is updated in place; NOT_CONVERGED / NAN keep the best finite state. */
hb_status hb_solve(hb_problem *p, const hb_solve_opts *o, hb_report *rep);
/* Harmonic coefficients of the current state (u* = E u, Eq. upghdft; reconstruction of Sec. 3.2). */
hb_status hb_get_harmonics(hb_problem *p, double *out);
/* Instance values of the current state [n_nodes][4][N]. */
hb_status hb_get_instances(hb_problem *p, double *out);

/* ---- hot-path entry points (host buffers; copies in and out are part of the call) ---------------- */

/* Residual r(y) of Eq. (Rmc) at instance values y (Dirichlet values taken from y as given): momentum
 * rows of Dirichlet nodes are 0.  precision 0 = FP64 kernels, 1 = FP32 kernels (inputs rounded). */
hb_status hb_residual(hb_problem *p, const double *y, double *r, int precision);
/* Jacobian-vector product at state y along v.  kind 0: the paper's tangent (P + C, Eqs. ptangent,
 * K_mat, ctangent, F_mat) with U and tau frozen at y; kind 1: the exact derivative of hb_residual;
 * kind 2: the paper's tangent assembled at y (Sec. 4's condensed storage, see hb_assemble_dev) and
 * applied as a sparse product (same operator as kind 0 up to rounding).
 * shift adds shift * M v on the velocity rows (pseudo time term, Sec. 2.3: shift = c1 rho / dt).
 * Dirichlet velocity rows return v (identity); v's Dirichlet velocity entries are treated as 0. */
hb_status hb_jv(hb_problem *p, const double *y, const double *v, double *jv, int kind, int precision,
                double shift);
/* The same product with FP32 host buffers (FP32 kernels): y, v, jv float [n_nodes][4][N].  Half the bytes
 * of hb_jv's FP64 buffers cross the host link; otherwise identical to hb_jv with precision 1. */
hb_status hb_jv_f32(hb_problem *p, const float *y, const float *v, float *jv, int kind, double shift);
/* Jacobi diagonal: diag(P) + shift M_AA (Sec. 2.3); 1 on Dirichlet velocity rows. */
hb_status hb_jacobi_diag(hb_problem *p, const double *y, double *d, int precision, double shift);

/* ---- device-pointer twins: all arrays on the problem's device, of type double (precision 0) or float
 * (precision 1), in instance layout; work is queued on `stream` (NULL: the problem's stream) and the
 * call returns without synchronising.  Outputs must not alias inputs. */
hb_status hb_residual_dev(hb_problem *p, const void *y, void *r, int precision, void *stream);
hb_status hb_jv_dev(hb_problem *p, const void *y, const void *v, void *jv, int kind, int precision,
                    double shift, void *stream);
/* Assemble the paper's tangent at the device state y (double for precision 0, float for 1): per node pair
 * and instance the blocks K, G, D, L of Eqs. (K_mat), (ctangent) with U and tau frozen at y, and per pair
 * the mass matrix (for the F block and the pseudo-time shift, applied as M (shift v + rho H v)); stored in
 * the problem (about 32 N bytes per node pair in FP32).  hb_jv_dev with kind 2 then applies the last
 * assembly (HB_ERR_STATE before one); the y argument of that call is used for the boundary terms. */
hb_status hb_assemble_dev(hb_problem *p, const void *y, int precision, void *stream);
hb_status hb_jacobi_diag_dev(hb_problem *p, const void *y, void *d, int precision, double shift,
                             void *stream);

/* Jacobian-vector product that allocates no device memory (the paper has no counterpart: this is a
 * library-integration entry point).  For callers that must not have the library allocate: an
 * application whose device memory is entirely owned by its own allocator (for example a framework's
 * caching pool, which can leave cudaMalloc failing while the pool still holds free memory), or a
 * latency-critical loop in which a cudaMalloc / cudaFree would stall it by synchronising the device.
 * Same arguments, layouts and result as hb_jv_dev.  Differences:
 *  - it performs no cudaMalloc, cudaFree or other allocating call; its only scratch (the per-outlet
 *    flow rates of resistance outlets) is a file-scope device array of 4096 doubles that every GPU
 *    which loads the library holds until the process exits;
 *  - outlets x instances above 4096 is rejected with HB_ERR_INVALID_ARG;
 *  - the boundary data must already be prepared: after the last hb_set_* boundary call (and after
 *    hb_set_launch_variant or hb_tune_patches), call one of hb_get_info, hb_residual*, hb_jv*,
 *    hb_jacobi_diag* or hb_solve once; otherwise HB_ERR_STATE;
 *  - the first call on a device looks up the scratch array's device address (cudaGetSymbolAddress, with
 *    that device current); make that first call before any stream capture;
 *  - all calls in the process share the one scratch array per device and it keeps the last call's
 *    contents (the call clears the part it uses before use): calls that overlap in time on the GPU,
 *    from any problem or stream, race on it and must be serialised by the caller;
 *  - it sums with atomics whatever hb_set_scatter says (the deterministic summation needs per-element
 *    slot buffers). */
hb_status hb_jv_dev_noalloc(hb_problem *p, const void *y, const void *v, void *jv, int kind, int precision,
                            double shift, void *stream);

/* ---- learned warm start (not the paper's method: Sec. 4 only suggests harmonic balance solutions as
 * machine-learning data) ---------------------------------------------------------------------------
 * A message-passing network over the mesh graph predicts the harmonic coefficients of the solution from
 * node positions, boundary flags, the inflow profile and the inflow waveform.  Weights are stored in
 * BF16, arithmetic is FP32.  Architecture, with mlp(X) = relu(X W1 + b1) W2 + b2:
 *   h = enc(x); for each layer: m_e = msg([h_src, h_dst, e_e]), a_i = sum_{e->i} m_e, h += upd([h, a]);
 *   out = dec(h), out = [n][4][2 n_h + 1] normalised harmonics (velocity / U, pressure relative to the
 *   mean outlet level / (p_scale rho U^2), U the largest mean inlet speed).
 * Parameters, flat FP32 (hb_mpnn_get_params): per MLP in the order enc, (msg_l, upd_l) for each layer,
 * dec: W1 [in][hidden], b1 [hidden], W2 [hidden][out], b2 [out], row-major. */
typedef struct hb_mpnn hb_mpnn;
typedef struct {
    int hidden;               /* 32 .. 64 */
    int layers;               /* message-passing layers, 1 .. 8 */
    int n_h;                  /* harmonics predicted; must equal the problems' n_h (<= 11) */
    int seed;                 /* initialisation seed */
    double p_scale;           /* pressure normalisation: (p - mean outlet level) / (p_scale rho U^2); <= 0
                                 means 1 */
} hb_mpnn_config;
/* Create a network with seeded parameters on `device`; INVALID_ARG for a config out of range (hidden
 * in [32, 64], layers in [1, 8], n_h in [0, 11]). */
hb_status hb_mpnn_create(const hb_mpnn_config *cfg, int device, hb_mpnn **out);
/* Free a network; NULL is accepted. */
hb_status hb_mpnn_destroy(hb_mpnn *net);
/* Forward MLP products on the tensor cores (default on; hidden 32 or 64): mma.sync TF32 with FP32
 * accumulation, the FP32 activations split into a TF32 head and tail against the BF16 weights (exact in
 * TF32), so the result keeps FP32 accuracy; 0 selects the FP32-FMA kernels.  INVALID_ARG for NULL. */
hb_status hb_mpnn_set_tensor_cores(hb_mpnn *net, int enable);
/* Number of FP32 parameters (the length of get/set and gradient arrays); 0 for NULL. */
int64_t hb_mpnn_num_params(const hb_mpnn *net);
hb_status hb_mpnn_get_params(hb_mpnn *net, float *params);          /* host [num_params] */
hb_status hb_mpnn_set_params(hb_mpnn *net, const float *params);    /* also resets the optimiser */
/* Mean squared error of the prediction against target harmonics (host, [n][4][2 n_h + 1], physical
 * units) and, if grad is non-NULL, its gradient with respect to the FP32 parameters (host). */
hb_status hb_mpnn_loss_grad(hb_mpnn *net, hb_problem *p, const double *target, float *loss, float *grad);
/* One Adam step (beta 0.9 / 0.999) on one problem's target harmonics; loss before the step. */
hb_status hb_mpnn_train_step(hb_mpnn *net, hb_problem *p, const double *target, float lr, float *loss);
/* Predicted harmonics [n][4][2 n_h + 1] in physical units (host). */
hb_status hb_mpnn_predict(hb_mpnn *net, hb_problem *p, double *harmonics);
/* The graph the network sees for a problem: node features x [n][32] (normalised position, wall /
 * inflow / outlet flags, inflow profile / its largest magnitude, inflow waveform series / |a0|, zero
 * padded), directed edges (both directions of every tetrahedron edge) and edge features e [n_edges][4]
 * (normalised offset, length).  Any output pointer may be NULL; *n_edges is always written. */
hb_status hb_mpnn_graph(hb_mpnn *net, hb_problem *p, float *x, int32_t *src, int32_t *dst, float *e,
                        int64_t *n_edges);
/* Set the problem's state to the prediction (Dirichlet values imposed on top). */
hb_status hb_mpnn_warm_start(hb_mpnn *net, hb_problem *p);
/* Attach a network (not owned) so that hb_solve with use_learned = 1 starts from its prediction and
 * with use_learned = 2 takes learned correction steps towards it. */
hb_status hb_attach_learned(hb_problem *p, hb_mpnn *net);

/* ---- time-domain march: the conventional solver the paper compares with (Sec. 3) ----------------------
 * GLS of Eq. (NS-weak) in the time domain (du/dt in place of H u, no least-squares time term) with
 * tau_hat of Eq. (tauhat), omega_hat = ||du/dt|| / ||u|| over the nodal velocities; generalized-alpha in
 * time (alpha_m = (3 - rho_inf) / (2 (1 + rho_inf)), alpha_f = 1 / (1 + rho_inf), gamma = 1/2 + alpha_m -
 * alpha_f; residual at (u, p)_{n+alpha_f} and du/dt_{n+alpha_m}); per step Newton on the paper's tangent
 * (+ c1 rho / dt M) with Jacobi-preconditioned GMRES.  It marches from rest (Dirichlet values at t = 0,
 * pressure at the mean outlet level) on a one-instance copy of the problem, with the Dirichlet and outlet
 * values evaluated from the problem's harmonic data at each time; the HB state of the problem is not
 * touched.  The state at the N instance times of the last period is kept for hb_get_march_samples. */
typedef struct {
    int precision;            /* 0: FP64 kernels; 1: FP32 Jacobian products, FP64 residual and Krylov   */
    int steps_per_period;     /* a multiple of N (the instance times are sampled); <= 0: 100 N         */
    int periods;              /* periods marched (4)                                                   */
    double rho_inf;           /* generalized-alpha spectral radius at infinite step (0.5)              */
    double newton_rtol;       /* per-step Newton stop on ||r|| / ||r_first|| (1e-3, as in Sec. 3)      */
    int newton_max;           /* Newton iterations per step (10)                                       */
    double gmres_rtol;        /* GMRES tolerance (0.03, as in Sec. 3)                                  */
    int gmres_restart;        /* (15)                                                                  */
    int max_gmres;            /* GMRES iteration cap per linear solve (300)                            */
    int tau_acceleration;     /* 1: tau_hat with omega_hat (Eq. tauhat); 0: tau of Eq. (tau)           */
    int verbose;              /* one line per instance time to stderr                                  */
} hb_march_opts;

typedef struct {
    int steps, newton_iters, gmres_iters, jv_calls;
    double seconds;
    double period_change;     /* ||u(t_end) - u(t_end - T)|| / ||u(t_end)|| (periods > 1)              */
    double max_newton_rel;    /* largest ||r|| / ||r_first|| left at the end of a step                 */
    int status;
} hb_march_report;

/* Fill the defaults: the paper's settings for its conventional solver (Sec. 3: GMRES 0.03, Newton 1e-3
 * per step), rho_inf = 0.5 (reading R13), 4 periods; INVALID_ARG for NULL. */
hb_status hb_default_march_opts(hb_march_opts *o);
/* HB_ERR_INVALID_ARG for bad options (steps_per_period not a multiple of N), HB_ERR_STATE without an
 * inflow, HB_ERR_NAN if the march produced non-finite values. */
hb_status hb_march(hb_problem *p, const hb_march_opts *o, hb_march_report *rep);
/* Hot-path entry points of the march (host buffers, one time level [n_nodes][4]): the residual at time
 * t (outlet levels at t; Dirichlet momentum rows 0; ydot's pressure column unused) and the paper tangent
 * (+ shift M on the velocity; Dirichlet rows identity on v) at y, both with tau_hat for the given
 * omega2 = omega_hat^2 (>= 0, else HB_ERR_INVALID_ARG). */
hb_status hb_time_residual(hb_problem *p, const double *y, const double *ydot, double *r, int precision, double t,
                           double omega2);
hb_status hb_time_jv(hb_problem *p, const double *y, const double *v, double *jv, int precision, double omega2,
                     double shift);
/* State of the last march at t_j = j T / N of its last period, [n_nodes][4][N] (the instance layout, so
 * it compares directly with hb_get_instances); HB_ERR_STATE before a march. */
hb_status hb_get_march_samples(hb_problem *p, double *out);

/* ---- batches of problems (many vessels of uneven size and N in one graph) ---------------------------
 * A batch applies the operator of every member problem in one captured CUDA graph (not the paper's
 * method: a throughput layer for many independent vessels).  In the default launch layout (2, see
 * hb_batch_set_grouping) the graph has 8 parallel branches, and each member's whole single-problem
 * operator -- output clearing, for the paper's tangent the node-level W = shift v + rho H v pass, the
 * element pass with the member's own launch variant and summation setting, the boundary terms -- runs on
 * branch q mod 8; the branches' launches run concurrently and fill one another's tails.  Layouts 0 and 1
 * instead run one persistent element pass over every member (or one per instance count) whose work items
 * (problem, patch) come from a global counter; they sum with atomics whatever hb_set_scatter says.
 * All problems must live on one device; their boundary data are prepared at creation.  The graph is
 * captured on first use and again whenever the operands, kind, shift or layout change, or a member's
 * boundary data or settings (backflow, stabilisation, summation, spectral path, launch variant,
 * patches) changed since the capture.  Work is ordered
 * after `stream` (NULL: the first problem's stream) and `stream` waits for it. */
typedef struct hb_batch hb_batch;
/* Create a batch over `count` problems (not owned; they must outlive the batch) at precision 0 or 1. */
hb_status hb_batch_create(hb_problem *const *problems, int count, int precision, hb_batch **out);
/* Free a batch (not its problems); NULL is accepted. */
hb_status hb_batch_destroy(hb_batch *b);
/* y[q], v[q], jv[q]: device arrays of problem q (double for precision 0, float for 1), instance
 * layout; same semantics as hb_jv_dev for each problem. */
hb_status hb_batch_jv_dev(hb_batch *b, const void *const *y, const void *const *v, void *const *jv, int kind,
                          double shift, void *stream);
/* Kernel launches queued by the batch since creation: its graph's launches times its replays (0 for
 * NULL). */
int64_t hb_batch_launch_count(const hb_batch *b);
/* Launch layout of the batch's graph: 0 one persistent element launch over every member (the kernel
 * dispatches on each work item's instance count); 1 one persistent element launch per instance count,
 * specialised for it, the launches on parallel graph branches (at most 8 distinct counts); 2 (default)
 * every member's single-problem operator (clearing, W pass, its own element launch, boundary terms) on
 * one of 8 parallel graph branches, members q, q + 8, ... in sequence on branch q mod 8, so that the
 * branches' launches fill one another's tails (the fastest: the element launches keep their arguments
 * in the constant bank, where 0 and 1 read each work item's arguments from shared memory).  Same results
 * in every layout up to the order of the atomic additions (a member set to deterministic summation keeps
 * it in layout 2).  The next hb_batch_jv_dev recaptures.  INVALID_ARG for a null batch or another
 * value. */
hb_status hb_batch_set_grouping(hb_batch *b, int grouping);
/* Patch-size autotuning: rebuild the problem's element patches (precision 0 or 1) with each candidate
 * node cap (and, for precision 1, each launch variant, see hb_set_launch_variant), time `reps`
 * paper-tangent Jv element passes with CUDA events, and keep the fastest.  Returns the chosen cap and
 * its time per pass (ms); the chosen variant is left set on the problem. */
hb_status hb_tune_patches(hb_problem *p, int precision, const int *candidates, int n_cand, int reps,
                          int *best_nl, double *best_ms);

/* ---- introspection ------------------------------------------------------------------------------ */
typedef struct {
    int64_t n_nodes, n_tets, n_faces, n_dirichlet_nodes, n_neumann_faces;
    int n_h, N, n_patches32, n_patches64, patch_nodes_max32, patch_elems_max32;
    int64_t device_bytes;
    double h_char;            /* edge of the regular tetrahedron of mean element volume (Sec. 2.3) */
    double u_ref;             /* largest mean inlet speed over the instances (CFL rule of Sec. 2.3)  */
    double p_ref;             /* mean outlet pressure level over outlets and instances              */
    int64_t assembled_pairs;  /* node pairs of the assembled tangent (0 before hb_assemble_dev)     */
} hb_info;
/* Sizes and derived quantities of a problem; also prepares pending boundary data (see
 * hb_jv_dev_noalloc). */
hb_status hb_get_info(hb_problem *p, hb_info *info);
/* Number of kernel launches queued by this problem since creation (all entry points). */
int64_t hb_launch_count(const hb_problem *p);
/* Launch variant of the FP32 paper-tangent element pass (no counterpart in the paper; a tuning knob):
 * 0 = 256 threads per block, two instances per thread on paired FP32 instructions; 1 = 384 threads,
 * one instance per thread (the default); 2 = 512 threads, one instance per thread; 3 = 192 threads, one
 * instance per thread, four resident blocks per SM (pays with patches small enough for four blocks'
 * shared memory, see hb_tune_patches); 4 = pipelined: one block per SM, 4 producer warps copy the next
 * patch's rows into a second shared-memory stage (16-byte asynchronous copies completing on an mbarrier)
 * while 20 consumer warps compute (one instance per thread); 5 = the same with 12 consumer warps on
 * instance pairs and paired FP32 instructions; 6 = as 4 with one producer warp issuing 1-D bulk copies.
 * Variants 4-6 need N = 9, 13 or 21 and the node-level W pass of hb_jv_dev (elsewhere, e.g. in
 * hb_jv_dev_noalloc and batches, they run variant 1).  All give the same operator up to FP32 rounding.  hb_tune_patches also searches it for precision 1.  HB_ERR_INVALID_ARG
 * for another value.  hb_get_launch_variant returns the current variant (-1 for a null problem). */
hb_status hb_set_launch_variant(hb_problem *p, int variant);
int hb_get_launch_variant(const hb_problem *p);
/* Implementation of the node-level spectral pass W = shift v + rho H v (the F block of Eq. F_mat and the
 * pseudo-time mass, a dense N x N product per node row) in FP32 at N = 9, 13, 21 (no counterpart in the
 * paper; a tuning knob): 0 = tcgen05 tensor cores with the accumulator in tensor memory, 1 = warp-level
 * mma.sync tensor cores, 2 = FP32 FMAs.  All are TF32 head/tail splits or FP32 and give the same W to FP32
 * accuracy; FP64 and other N always use the FMA form.  HB_ERR_INVALID_ARG for another value;
 * hb_get_spectral_path returns the current path (-1 for a null problem). */
hb_status hb_set_spectral_path(hb_problem *p, int path);
int hb_get_spectral_path(const hb_problem *p);
/* Element-kernel timing: when enabled, every launch of the fused element kernel is bracketed by CUDA
 * events on the stream it is launched on.  hb_profile_read synchronises with those events, returns the
 * summed device time in milliseconds and the number of launches since the last read, and resets. */
hb_status hb_profile_elem(hb_problem *p, int enable);
hb_status hb_profile_read(hb_problem *p, double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* HBGLS_H */
