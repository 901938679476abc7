/*
 * lbe.h -- C ABI of the GB300 Lattice Boltzmann Electrokinetics library with
 * constant-potential (metallic) electrodes.
 *
 * Method: Asta, Palaia, Trizac, Levesque, Rotenberg, "Lattice Boltzmann
 * Electrokinetics simulation of nanocapacitors", arXiv:1907.04732.
 *
 * Units are lattice units: spacing = time step = 1, k_B T = e = 1.  Potentials
 * are reduced (phi = beta e psi), concentrations are solute amounts per node
 * (n_k = rho_k dx^3), charges are in units of e.
 *
 * Lattice layout: node r = x + nx*(y + ny*z), 0 <= x < nx etc.  Per-node
 * fields are arrays of N = nx*ny*nz values; multi-component fields are
 * component-major ([k][r] for species, [a][r] for vector components).
 *
 * Ownership: a handle owns all of its device state (allocated in lbe_create /
 * lbe_set_geometry, freed in lbe_destroy).  Every buffer passed in or out is
 * owned by the caller; a flag says whether it lives in host or device memory.
 * All work is ordered on the CUDA stream given to lbe_create (NULL = the
 * legacy default stream).  Calls that return data to host memory synchronise
 * that stream; lbe_step synchronises only to test Poisson convergence.
 *
 * Errors: every function returns LBE_OK (0) or a negative LBE_ERR_* code; the
 * message of the last error on a handle is lbe_last_error(handle).  No call
 * aborts the process.  A CUDA error is reported as LBE_ERR_CUDA and leaves
 * the handle unusable except for lbe_destroy.
 */
#ifndef LBE_H
#define LBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBE_OK 0
#define LBE_ERR_ARG (-1)        /* invalid argument or size */
#define LBE_ERR_CUDA (-2)       /* a CUDA call failed */
#define LBE_ERR_NOCONVERGE (-3) /* Poisson solve hit poisson_max_iter */
#define LBE_ERR_NONFINITE (-4)  /* NaN/Inf met in a reduction */
#define LBE_ERR_STATE (-5)      /* call out of order (e.g. step before init) */
#define LBE_ERR_GEOMETRY (-6)   /* fluid node on a non-periodic face, bad id */

#define LBE_FP64 0 /* all state and arithmetic in FP64 */
#define LBE_FP32 1 /* FP32 deviations from the rest state, int64 fixed-point
                      solute and potential (units rho_b 2^-40 and 2^-48;
                      |potential| < 100), the Poisson residual summed
                      exactly in integers, FP64 reductions */

#define LBE_RULE_MIDPLANE 0 /* lbe_params.boundary_rule */
#define LBE_RULE_NODE 1

#define LBE_MAX_SPECIES 4
#define LBE_MAX_ELECTRODES 16

/* lbe_fields selectors */
#define LBE_FIELD_PHI 0 /* reduced potential, N doubles */
#define LBE_FIELD_N 1   /* solute amounts, nspecies*N doubles */
#define LBE_FIELD_RHO 2 /* solvent density, N doubles (0 on solid nodes) */
#define LBE_FIELD_U 3   /* solvent velocity (sum f c + F/2)/rho, 3*N doubles */
#define LBE_FIELD_F 4   /* populations after streaming, 19*N doubles, in the
                           velocity order c_0 = (0,0,0);
                           c_1..c_9 = (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0)
                           (1,0,1) (1,0,-1) (0,1,1) (0,1,-1); c_{i+9} = -c_i */
#define LBE_FIELD_QNODE 5 /* induced charge of each electrode node, N doubles:
                             the node's term of Eq. Qelec (links to fluid,
                             doubled weights); 0 on fluid nodes.  Summed over
                             the nodes of electrode e it is Q_e. */

typedef struct lbe_handle lbe_handle;

typedef struct {
  int nx, ny, nz;       /* lattice size (Sec. "Parallel plate capacitor");
                           nx*ny*nz < 2^31 */
  int periodic[3];      /* 1 = periodic along x/y/z; a non-periodic face must
                           be solid (its nodes are electrode nodes) */
  double tau;           /* BGK relaxation time, Eq. LBpop (nu = (tau-1/2)/3) */
  double bjerrum;       /* Bjerrum length l_B in lattice units, Eq. lambda */
  int nspecies;         /* ionic species, 1..LBE_MAX_SPECIES */
  double z[LBE_MAX_SPECIES];        /* valencies z_k (integers, |z| <= 4) */
  double D[LBE_MAX_SPECIES];        /* diffusivities D_k, Eq. NP */
  double rho_bulk[LBE_MAX_SPECIES]; /* initial uniform concentrations */
  double e_app[3];      /* applied field beta e E dx (Sec. "Electrokinetic
                           effects"), enters the link chemical-potential
                           differences */
  int flow;             /* 1: solvent evolves (LB + advection);
                           0: solvent at rest (pure Poisson-Nernst-Planck) */
  int precision;        /* LBE_FP64 or LBE_FP32 */
  double poisson_tol;   /* stop when max_r |residual(r)|/diag(r) <= tol */
  int poisson_max_iter; /* iteration cap per Poisson solve */
  int boundary_rule;    /* LBE_RULE_MIDPLANE (default): the paper's rule, Eq.
                           DiscreteLaplacianModif (links to solid doubled, the
                           interface half-way between solid and fluid nodes);
                           LBE_RULE_NODE: the first-order rule the paper starts
                           from in Sec. "Imposing conducting boundary
                           conditions" (plain Eq. DiscreteLaplacian, solid
                           nodes held at their potential), for comparison;
                           FP64 form only (LBE_ERR_ARG otherwise) */
} lbe_params;

/* Defaults: 1x1x1, periodic, tau 1, l_B 1, 1:1 salt with D = 0.05 and
 * rho = 0.01, no field, flow on, FP64, tol 1e-13, 100000 iterations, the
 * paper's boundary rule. */
void lbe_default_params(lbe_params *p);

/* Create a lattice.  cuda_stream is a cudaStream_t (may be NULL).  On
 * success *out receives the handle. */
int lbe_create(const lbe_params *p, void *cuda_stream, lbe_handle **out);

/* Free all device state of the handle (NULL is accepted). */
int lbe_destroy(lbe_handle *h);

/* Message of the last error on h (static string if h is NULL). */
const char *lbe_last_error(const lbe_handle *h);

/* Geometry (Sec. "Imposing conducting boundary conditions": chi_s, and the
 * electrode regions of Figs. 2 and 7).  node_id has N bytes: 0 = fluid node,
 * e in 1..n_electrodes = solid node of electrode e.  on_device selects where
 * node_id lives.  Fails with LBE_ERR_GEOMETRY if an id exceeds n_electrodes
 * or a fluid node lies on a non-periodic face.  In the FP32 form it also
 * builds the multigrid hierarchy of the Poisson preconditioner and inverts
 * its coarsest operator on the host (synchronising the stream). */
int lbe_set_geometry(lbe_handle *h, const uint8_t *node_id, int n_electrodes, int on_device);

/* Electrode potentials psi_e (reduced, host array of n_electrodes doubles).
 * Only differences matter (Sec. "Parallel plate capacitor").  After lbe_init
 * the potential is re-solved at once so that the state stays consistent;
 * potentials equal to the current ones are uploaded and nothing else is done
 * (the state is already consistent).  Non-finite values, and in the FP32
 * form values of magnitude 100 or more (its fixed-point range), fail with
 * LBE_ERR_ARG. */
int lbe_set_voltage(lbe_handle *h, const double *psi);

/* Initial state (Sec. "Potential and concentration profiles"): uncharged
 * capacitor, n_k = rho_bulk on fluid nodes, solvent at rest with unit
 * density, potential = Laplace solution for the applied voltage. */
int lbe_init(lbe_handle *h);

/* Advance nsteps LBE time steps.  One step: link fluxes of Eq. LF2 and the
 * solvent force, BGK collision with forcing (Eq. LBpop) and streaming with
 * bounce-back, advection, then the Poisson solve of Eq. SOR's fixed point
 * with the modified Laplacian of Eq. DiscreteLaplacianModif, started from
 * the extrapolation in time of the previous steps' potentials (the converged
 * potential does not depend on the start).  The steps of one call run
 * without host synchronisation, except that the solves' status is read
 * every 1024 steps (a failed solve ends the call there) and at the end.
 * Returns LBE_ERR_NOCONVERGE if a Poisson solve reached poisson_max_iter or
 * a refinement round failed to halve the residual (a tolerance below what
 * the form's arithmetic resolves). */
int lbe_step(lbe_handle *h, int nsteps);

/* Induced charge of every electrode, Eq. Qelec, from the current potential:
 * Q_e = -(1/(4 pi l_B)) sum over nodes of electrode e of the modified
 * Laplacian, taken over links to fluid nodes.  q_out receives n_electrodes
 * doubles in host (out_on_device = 0) or device memory.  FP64 reduction in a
 * fixed order (bitwise reproducible). */
int lbe_induced_charge(lbe_handle *h, double *q_out, int out_on_device);

/* Copy one field (LBE_FIELD_*) of the current state into out as doubles. */
int lbe_fields(lbe_handle *h, int which, void *out, int out_on_device);

/* Overwrite the solute amounts (nspecies*N doubles) and/or the potential
 * (N doubles) of an initialised lattice; either pointer may be NULL.  The
 * potential on solid nodes is reset to the electrode potentials.  In the
 * FP32 form, amounts and potentials outside its fixed-point ranges (or
 * non-finite) return LBE_ERR_NONFINITE. */
int lbe_set_state(lbe_handle *h, const double *n, const double *phi, int on_device);

/* Checkpoint: the complete dynamic state (including the earlier potentials
 * the next solve extrapolates from) as an opaque blob, every array in the
 * form's own types, so that a restart continues bit for bit.  With blob
 * NULL, *size receives the needed size.  lbe_load_state restores a blob
 * written by a handle with the same parameters and geometry, built with the
 * same extrapolation order and blob format. */
int lbe_save_state(lbe_handle *h, void *blob, size_t *size);
int lbe_load_state(lbe_handle *h, const void *blob, size_t size);

/* Statistics of the most recent lbe_init/lbe_step call. */
typedef struct {
  long long poisson_iters;      /* CG iterations summed over the call's solves */
  int poisson_solves;           /* Poisson solves in the call */
  int poisson_max_iters;        /* largest single solve */
  double poisson_residual;      /* final max |res|/diag of the last solve */
} lbe_stats;
int lbe_get_stats(const lbe_handle *h, lbe_stats *out);

/* Induced charge of every electrode (the same quantity as
 * lbe_induced_charge) from buffers the caller owns, without allocating any
 * device memory.  (The paper has no counterpart: this entry point exists for
 * callers that cannot allocate -- code whose device memory all comes from its
 * own pool or budget, or that must not allocate while it is recording work,
 * for instance during CUDA stream capture.)
 *   phi      device, N doubles: potential of every node (solid nodes hold
 *            their electrode potential), layout as lbe_fields(LBE_FIELD_PHI)
 *   node_id  device, N bytes: 0 fluid, e = 1..n_electrodes electrode e; an
 *            id above n_electrodes is not checked: such a node counts as
 *            solid for its neighbours and its own charge is not reported
 *   nx,ny,nz lattice size (nx*ny*nz < 2^31); periodic[3] host flags
 *   bjerrum  l_B > 0; q_out device, n_electrodes doubles (written)
 *   cuda_stream  stream the work is ordered on (NULL = legacy stream)
 * Scratch: the per-block partial sums use a fixed device array of 128 KiB
 * (1024 blocks x LBE_MAX_ELECTRODES doubles) that every GPU which loads this
 * library keeps until the process exits; any lattice size fits it, while
 * n_electrodes above LBE_MAX_ELECTRODES is rejected with LBE_ERR_ARG.  The
 * first call on a device looks up that array's device address (and caches
 * it for the life of the process), so make that first call outside any
 * stream capture, and do not reset the device (cudaDeviceReset) between
 * calls: the cached address would then be stale.  Every call
 * rewrites the partials it reads, but all calls share the one array: calls
 * that can overlap on the GPU (different streams, or threads without
 * ordering) race and must be serialised by the caller.  Returns LBE_OK,
 * LBE_ERR_ARG or LBE_ERR_CUDA; the message is lbe_last_error(NULL) on the
 * calling thread.  Asynchronous: q_out is ready when the stream has run. */
int lbe_induced_charge_static(const double *phi, const uint8_t *node_id, int nx, int ny, int nz,
                              const int *periodic, double bjerrum, int n_electrodes, double *q_out,
                              void *cuda_stream);

/* Device time per phase of the lbe_step calls made between
 * lbe_profile_begin and lbe_profile_end, from CUDA events recorded on the
 * handle's stream around each phase (a measurement aid; results unchanged). */
typedef struct {
  double sweep_ms;             /* fused flux + collide-stream kernel */
  long long sweep_launches;
  double advect_ms;            /* advection kernel */
  long long advect_launches;
  double poisson_ms;           /* whole Poisson solves */
  long long poisson_solves;
  long long poisson_iters;
  long long kernel_launches;   /* every kernel launched by the profiled steps */
} lbe_profile;
int lbe_profile_begin(lbe_handle *h);
int lbe_profile_end(lbe_handle *h, lbe_profile *out);

/* ------------------------------------------------------------------------
 * Batched FP32 form: many independent lattices ("instances", each with its
 * own size, geometry, voltages, Debye length and diffusivities) advanced
 * together.  The instances' state is concatenated in device memory; every
 * kernel of a step is one persistent launch over all instances (tiles of 1024
 * consecutive nodes of one instance), and a whole step -- fused flux and
 * collide-stream sweep, advection, Poisson solve with per-instance
 * convergence -- runs as one CUDA graph launch.  The arithmetic per node is
 * that of LBE_FP32 on a single lattice; results match a single-lattice
 * LBE_FP32 run of each instance up to the Poisson stopping point.
 *
 * Restrictions: precision LBE_FP32; a 1:1 monovalent salt (nspecies 2,
 * z = +1, -1, equal rho_bulk); flow, poisson_tol and poisson_max_iter equal
 * for all instances; at most LBE_BATCH_MAX_ELECTRODES electrodes per
 * instance; total node count < 2^31.  Other violations return LBE_ERR_ARG.
 * ------------------------------------------------------------------------ */
#define LBE_BATCH_MAX_ELECTRODES 4
typedef struct lbe_batch lbe_batch;

/* Create a batch of n instances from params[0..n-1] (host).  cuda_stream as
 * for lbe_create (NULL: the batch creates and owns a stream). */
int lbe_batch_create(const lbe_params *params, int n, void *cuda_stream, lbe_batch **out);
int lbe_batch_destroy(lbe_batch *b);
/* Message of the last error on b (or for b == NULL). */
const char *lbe_batch_last_error(const lbe_batch *b);
/* Geometry of instance i: node_id host, N_i bytes, as lbe_set_geometry. */
int lbe_batch_set_geometry(lbe_batch *b, int i, const uint8_t *node_id, int n_electrodes);
/* Potentials of instance i's electrodes: psi host, n_electrodes doubles.
 * Before lbe_batch_init (LBE_ERR_STATE after). */
int lbe_batch_set_voltage(lbe_batch *b, int i, const double *psi);
/* Equilibrium start of every instance (as lbe_init), the multigrid
 * hierarchies (with each coarsest operator inverted on the host where it is
 * positive definite), the persistent grid picked by timing candidate grids
 * (autotuner), and the first Poisson solves.  Every instance needs a
 * geometry first. */
int lbe_batch_init(lbe_batch *b);
/* nsteps time steps of every instance; synchronises once at the end to read
 * the Poisson status (LBE_ERR_NOCONVERGE / LBE_ERR_NONFINITE if any
 * instance failed). */
int lbe_batch_step(lbe_batch *b, int nsteps);
/* Induced charge of every electrode of every instance (Eq. of the induced
 * charge, FP64 reductions in a fixed order): q_out receives
 * n * LBE_BATCH_MAX_ELECTRODES doubles, [i][e], zero past an instance's
 * electrode count; host or device memory by out_on_device. */
int lbe_batch_charge(lbe_batch *b, double *q_out, int out_on_device);
/* Field of instance i: LBE_FIELD_PHI (N_i doubles) or LBE_FIELD_N
 * (2*N_i doubles), layout as lbe_fields. */
int lbe_batch_fields(lbe_batch *b, int i, int which, double *out, int out_on_device);
/* lbe_stats of the last init/step call; poisson_iters sums CG iterations
 * over instances, poisson_max_iters is the most iterations of one solve of
 * one instance. */
int lbe_batch_get_stats(const lbe_batch *b, lbe_stats *out);
/* Device time per phase of the lbe_batch_step calls made between
 * lbe_batch_profile_begin and lbe_batch_profile_end (events recorded around
 * the sweep, the advection and the Poisson solve of every step; each step is
 * then waited for).  poisson_iters sums CG iterations over instances;
 * kernel_launches is counted with LBE_POISSON_GRAPH=0 only (else -1). */
int lbe_batch_profile_begin(lbe_batch *b);
int lbe_batch_profile_end(lbe_batch *b, lbe_profile *out);
/* Autotuner outcome: the persistent grid (blocks) in use, and the measured
 * sweep time (ms) of each of the LBE_BATCH_TUNE_CANDIDATES candidate grids
 * of k * SM-count blocks, k = 1, 2, 3, 4, 6, 8 (ms_out may be NULL). */
#define LBE_BATCH_TUNE_CANDIDATES 6
int lbe_batch_tuning(const lbe_batch *b, int *grid_blocks, double *ms_out);

/* ------------------------------------------------------------------------
 * Reverse-mode derivative (adjoint) of the induced charge after T steps of
 * the FP32 form with the solvent at rest (flow = 0; a 1:1 salt with one
 * bulk concentration).  The objective is S = sum_e dq[e] Q_e(T) (Eq. Qelec);
 * its gradient is returned with respect to the electrode potentials, the
 * bulk concentration rho_b (the Debye length enters only through it:
 * rho_b = 1 / (8 pi l_B lambda_D^2)), the ion diffusivities and a soft
 * electrode occupancy chi per node.  The occupancy derivative is that of a
 * continuous reading of the method which equals it at chi in {0, 1}: the
 * Poisson row of node r is (1 - chi_r)(lap phi + 4 pi l_B rho_el) +
 * chi_r (psi - phi_r) with link factor 1 + (chi_r - chi_j)^2 (the doubling
 * of fluid-solid links of Eq. DiscreteLaplacianModif), an ion link carries
 * the flux of Eq. LF2 times (1 - chi_r)(1 - chi_j), the initial ions are
 * rho_b (1 - chi), and Q_e sums chi_r (1 - chi_j) over the modified-Laplacian
 * links of electrode-e nodes.  It is evaluated at the handle's (binary)
 * geometry; a fluid node's chi turns it into part of soft_electrode.
 * ------------------------------------------------------------------------ */
typedef struct {
  double dpsi[LBE_MAX_ELECTRODES]; /* dS/dpsi_e */
  double drho_bulk;                /* dS/drho_b */
  double dD[LBE_MAX_SPECIES];      /* dS/dD_k (species order of lbe_params) */
  long long poisson_iters;         /* CG iterations of the adjoint Poisson solves */
  long long recomputed_steps;      /* forward steps recomputed from checkpoints */
  double recompute_ms;             /* device time: forward recomputation */
  double flux_ms;                  /* device time: transposed flux steps */
  double solve_ms;                 /* device time: adjoint Poisson solves */
} lbe_adjoint_grad;

/* Forward pass for a later lbe_adjoint_backward: lbe_init, then nsteps
 * steps, keeping the state every checkpoint_every steps in device memory
 * (48 bytes per node per checkpoint: solute, potential and the warm start's
 * three earlier potentials; plus 20 bytes per node per step of one segment
 * during the backward pass).  q_out (host, n_electrodes doubles, may be
 * NULL) receives Q(T).  LBE_ERR_STATE when the handle is not an FP32,
 * flow-off, 1:1-salt lattice with a geometry. */
int lbe_adjoint_forward(lbe_handle *h, int nsteps, int checkpoint_every, double *q_out);

/* The same forward pass with the checkpoints placed by the binomial schedule
 * of Griewank and Walther ("revolve") within device_bytes of checkpoint
 * memory (48 bytes per node per checkpoint slot; at least two slots, the
 * initial and the final state; LBE_ERR_ARG below).  With s = slots - 2 the
 * backward pass recomputes every forward step at most r times, r the
 * smallest integer with C(s + r, s) >= nsteps, and keeps no per-step states;
 * the gradient is bitwise that of lbe_adjoint_forward.  The schedule's
 * first checkpoints are taken during this pass, so its steps are reused. */
int lbe_adjoint_forward_budget(lbe_handle *h, int nsteps, size_t device_bytes, double *q_out);

/* Backward pass of the last lbe_adjoint_forward (LBE_ERR_STATE if the state
 * changed since): dq (host, n_electrodes weights), soft_electrode in
 * 1..n_electrodes, out receives the parameter gradients, dchi (N doubles,
 * host or device by dchi_on_device, may be NULL) the occupancy gradient.
 * Recomputes the forward states segment by segment and leaves the handle in
 * the forward pass's final state. */
int lbe_adjoint_backward(lbe_handle *h, const double *dq, int soft_electrode, lbe_adjoint_grad *out, double *dchi,
                         int dchi_on_device);

#ifdef __cplusplus
}
#endif

#endif /* LBE_H */
