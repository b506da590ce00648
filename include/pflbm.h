/*
 * pflbm.h -- C interface of the GB300 conservative Allen-Cahn phase-field
 * lattice Boltzmann method (PFLBM) library, libpflbm.so.
 *
 * The method (section "Conservative Allen-Cahn model" of Schwarzmeier et al.,
 * "Comparison of free-surface and conservative Allen-Cahn phase-field lattice
 * Boltzmann method"):
 *   - phase-field PDFs h_i on D3Q15 (or D3Q27, pfl_params.h_lattice) with
 *     phi = sum_i h_i (Eq. zeroth_moment_phase),
 *     relaxation time tau_phi = M / c_s^2 (Eq. pflbm-tau, read as the shifted
 *     time: omega_phi = 1 / (3 M + 1/2)) and the Allen-Cahn forcing
 *     F^phi = 4 phi (1 - phi) / xi * n applied with Guo's scheme;
 *   - hydrodynamic PDFs g_i on D3Q27 with normalised pressure p* = sum_i g_i
 *     (Eq. zeroth_moment_hydro), incompressible equilibrium (Eq. feq with
 *     rho_0 = 1), forces F = F_s + F_b + F_p + F_mu;
 *   - rho(phi) and tau(phi) linearly interpolated between the phases;
 *   - weighted-orthogonal MRT collision (Eq. mrt) fused with streaming (Eq. LBE).
 *
 * Conventions
 *   - Cells are x-fastest: cell = x + nx * (y + ny * z).  Scalar fields are N
 *     doubles, vector fields are 3N doubles SoA (all x, then all y, then all z).
 *   - Population order ("canonical"): loop cz, cy, cx over -1, 0, 1 with cx
 *     fastest; D3Q27 keeps all 27 (index 9(cz+1) + 3(cy+1) + (cx+1)), D3Q15
 *     keeps the 15 with |c|^2 in {0, 1, 3}.  Populations are SoA [i][cell].
 *   - Faces are ordered -x, +x, -y, +y, -z, +z.  Both faces of one axis must
 *     carry the same kind.  No-slip faces use halfway bounce-back; the phi
 *     stencil mirrors phi across them.
 *   - Heavy phase phi = 1 (rho_h), light phase phi = 0 (rho_l).
 *   - All device work is queued on the stream passed to pfl_init; calls that
 *     return data to the host synchronise that stream.
 *   - A context lives on the device that holds its workspace.  Each call makes
 *     that device current while it runs and gives the caller's current device
 *     back before it returns, on every path; a NULL stream is that device's
 *     legacy default stream.  The same holds for batches.
 *
 * Memory ownership: the library never allocates device memory.  The caller
 * allocates one device buffer of pfl_workspace_bytes() bytes (for example a
 * torch uint8 tensor), passes it to pfl_init and keeps it alive until
 * pfl_destroy.  The context itself is a small host object owned by the library.
 *
 * Errors: every call returns a pfl_status.  PFL_ERR_ARG leaves the context
 * untouched; PFL_ERR_CUDA means a CUDA call failed (the context should be
 * destroyed); pfl_last_error() returns a message for the calling thread.
 */
#ifndef PFLBM_H
#define PFLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfl_ctx pfl_ctx;

/* Largest flow speed |u| (lattice units) that pfl_diag accepts.  The LBM
 * equilibria are expansions in u / c_s (Eq. feq); beyond |u| = 0.3
 * (u / c_s = 0.52) a run is taken as unstable, like one with NaN/Inf. */
#define PFL_SPEED_LIMIT 0.3

typedef enum {
  PFL_OK = 0,
  PFL_ERR_ARG = 1,      /* invalid argument or parameter set                  */
  PFL_ERR_CUDA = 2,     /* a CUDA runtime call failed                          */
  PFL_ERR_OOM = 3,      /* workspace too small                                 */
  PFL_ERR_UNSTABLE = 4, /* the last diagnostic found NaN/Inf in phi or a flow
                         * speed above PFL_SPEED_LIMIT                          */
  PFL_ERR_STATE = 5     /* call not valid in the context's current state       */
} pfl_status;

/* Storage precision of the populations.  PFL_FP64: FP64 storage and arithmetic
 * (reference mode).  PFL_FP32: FP32 storage and arithmetic.  PFL_FP16S
 * (shifted FP16 storage): each population is stored in FP16 as its deviation
 * from the rest equilibrium of the cell that wrote it -- h_i from w_i phi,
 * g_i from w_i P with P = fp16(p*) kept per cell -- divided by its lattice
 * weight and scaled by a power of two; arithmetic in FP32; phi kept in FP32.
 * The initial state is stored against its own phi0 and p0, exactly for a
 * fluid at rest. */
typedef enum { PFL_FP64 = 0, PFL_FP32 = 1, PFL_FP16S = 2 } pfl_precision;

typedef enum { PFL_PERIODIC = 0, PFL_NOSLIP = 1 } pfl_bc;

/* PFL_MRT: weighted-orthogonal MRT (degree-2 moments of g at omega(phi), of h
 * at omega_phi together with degree 1; all higher moments at rate 1).
 * PFL_BGK: single rate per lattice (Eq. BGK), a special case kept for testing. */
typedef enum { PFL_MRT = 0, PFL_BGK = 1 } pfl_collision;

typedef struct {
  int nx, ny, nz;      /* lattice cells, each >= 1                                  */
  int bc[6];           /* pfl_bc per face -x,+x,-y,+y,-z,+z                          */
  double rho_h, rho_l; /* phase densities (> 0), rho_h is the reference density     */
  double nu_h, nu_l;   /* kinematic viscosities; tau = 3 nu + 1/2 per phase (Eq. kin-viscosity) */
  double sigma;        /* surface tension (>= 0)                                     */
  double mobility;     /* M > 0                                                      */
  double xi;           /* interface width (> 0), lattice units                       */
  double gravity[3];   /* body-force acceleration g, F_b = rho g                      */
  int precision;       /* pfl_precision                                              */
  int collision;       /* pfl_collision                                              */
  int engine;          /* pfl_engine                                                 */
  int h_lattice;       /* phase-field lattice: 15 (D3Q15; also when 0) or 27 (D3Q27, the
                        * paper's own 3-D choice); 9 selects the paper's 2-D lattices,
                        * D2Q9 for h and g, and needs nz = 1 with periodic z faces.
                        * The collisions keep their moment form on every lattice. */
  int solids;          /* 1: the lattice may hold solid cells (pfl_set_solid; 4 bytes
                        * per cell of workspace; fused engine only), 0: none */
  int hydrostatic;     /* 1: pfl_init called with p0 == NULL starts from the pressure of
                        * the fluid at rest under gravity (the paper's start in its
                        * gravity cases, sections "Gravity wave", "Rising bubble",
                        * "Drop impact"); gravity must then act along one axis.
                        * 0: p* starts at zero unless p0 is given. */
  double p_level;      /* hydrostatic start: cell-centre coordinate along the gravity
                        * axis where the pressure is zero */
} pfl_params;

/* How a single lattice is stepped.  PFL_ENGINE_AUTO: the fused two-array step
 * (stream-collide and phi stencil in one launch, populations in two array
 * pairs) for the MRT collision on lattices with 27 N < 2^32, else the in-place
 * one.  PFL_ENGINE_INPLACE: one array pair updated in place (AA pattern) and a
 * separate phi = sum h pass.  Both give the same results. */
typedef enum { PFL_ENGINE_AUTO = 0, PFL_ENGINE_INPLACE = 1 } pfl_engine;

/* Device bytes the workspace must hold for these parameters (0 if invalid). */
size_t pfl_workspace_bytes(const pfl_params* p);

/* The hydrostatic start of pfl_init, on the host: the normalised pressure
 * p* = p / (rho(phi0) c_s^2) of the fluid at rest under gravity, from which
 * the paper starts its gravity cases (sections "Gravity wave", "Rising
 * bubble", "Drop impact").  The same numbers pfl_init uses with
 * pfl_params.hydrostatic = 1 and p0 == NULL: along every line of cells
 * parallel to the gravity axis s, dp/ds = rho(phi0) g_s integrated by the
 * trapezoid rule between cell centres, p = 0 at s = p->p_level (linear
 * interpolation between the two cells around it).  A caller can inspect or
 * amend it (a bubble's Laplace jump, another gauge) and pass it as p0.
 *   phi0: N host doubles, x-fastest; pstar: N host doubles, written.
 * Needs no GPU and no context; p->hydrostatic is not read.  PFL_ERR_ARG for
 * NULL or device arrays, invalid parameters, gravity not along exactly one
 * axis, or a non-finite p_level. */
pfl_status pfl_hydrostatic_pstar(const pfl_params* p, const double* phi0, double* pstar);

/* Create a context and write the initial state.
 *   phi0: N doubles, required.  u0: 3N doubles SoA or NULL (zero).  p0: N
 *   doubles of initial normalised pressure p* or NULL: zero, or with
 *   pfl_params.hydrostatic = 1 the hydrostatic p* = p / (rho(phi0) c_s^2) with
 *   dp/ds = rho(phi0) g_s integrated along each line of cells parallel to the
 *   gravity axis s (trapezoid rule between cell centres, FP64 on the host) and
 *   p = 0 at s = p_level (linear interpolation between the two cells around
 *   it).  A given p0 overrides the hydrostatic start.  Each may be a host or a
 *   device pointer.  The populations start at their equilibria
 *   h^eq(phi0, u0) and g^eq(p0, u0); phi is then recomputed as sum_i h_i.
 *   workspace: device pointer, >= pfl_workspace_bytes(p) bytes, 256-byte aligned.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * Rejects (PFL_ERR_ARG) omega_h, omega_l or omega_phi outside (0, 2), M <= 0,
 * xi <= 0, densities <= 0, dims < 1, mixed face kinds on one axis. */
pfl_status pfl_init(const pfl_params* p, const double* phi0, const double* u0, const double* p0,
                    void* workspace, size_t workspace_bytes, void* stream, pfl_ctx** out);

/* Advance n_steps >= 0 time steps.  Asynchronous: only queues kernels.
 * The fused engine advances whole runs of graph_k steps (default 32) by
 * replaying a CUDA graph of them, captured on first use on a stream of the
 * context's own; the rest, and every step while the caller's stream is being
 * captured, launch one by one.  Both give bitwise the same states. */
pfl_status pfl_step(pfl_ctx* ctx, int n_steps);

/* Steps per CUDA graph of the fused engine: 0 (launch every step on its own)
 * or even in [2, 4096].  Drops the graphs captured so far.  Synchronises the
 * stream.  PFL_ERR_ARG for other values. */
pfl_status pfl_set_graph_steps(pfl_ctx* ctx, int graph_steps);

/* Macroscopic fields at the current time: phi, rho(phi), p = p* rho c_s^2
 * (Eq. zeroth_moment_hydro and the definition of p*) and u = sum_i c_i g_i +
 * F / (2 rho) (3N SoA).  Any pointer may be NULL; each may be host or device.
 * Synchronises the stream. */
pfl_status pfl_fields(pfl_ctx* ctx, double* phi, double* rho, double* p, double* u);

/* Populations at the current time in canonical order and layout, converted to
 * FP64: h is QN (Q = 15, 27 or 9, the h lattice), g is 27N doubles (9N on the
 * 2-D lattices; either may be NULL; host or device).
 * Synchronises. */
pfl_status pfl_populations(pfl_ctx* ctx, double* h, double* g);

/* Overwrite the populations (canonical order, FP64, host or device; rounded
 * to the storage precision) and recompute phi.  Synchronises. */
pfl_status pfl_set_populations(pfl_ctx* ctx, const double* h, const double* g);

/* Solid cells inside the lattice, voxelised obstacles and channel walls (the
 * Taylor bubble's pipe, section "Taylor bubble": no-slip walls on a Cartesian
 * grid).  mask: N bytes (host or device), nonzero = solid.  A link from a
 * fluid cell into a solid one is bounced back half-way, as at a no-slip face;
 * a phi stencil read of a solid neighbour returns the cell's own phi (neutral
 * wetting); solid cells are not updated, hold zero populations, and every
 * pfl_fields output is zero there.  Needs pfl_params.solids = 1 at init and
 * comes before the first step (PFL_ERR_STATE otherwise).  The adjoint and the
 * batch engine do not take solid cells.  Synchronises. */
pfl_status pfl_set_solid(pfl_ctx* ctx, const unsigned char* mask);

/* Saved states (checkpoint and resume).  A state is the stored arrays of the
 * context as they are (the current h and g in the storage precision, both phi
 * buffers, the link words of solid cells, the FP16S p* shifts) after a small header with the
 * lattice, the engine, the step count and the layout flags.  Loading it into a
 * context of the same lattice, boundaries, precision, phase-field lattice and
 * engine resumes the run bitwise: the step count (and with it the FP16
 * rounding seeds) continues.  The physical parameters of the loading context
 * apply from then on.
 *   pfl_state_bytes: bytes of a saved state of this context (0 if ctx is NULL).
 *   pfl_save: writes the state to buf (host or device, >= pfl_state_bytes).
 *   pfl_load: reads it back; PFL_ERR_ARG for a buffer that is short, not a
 *     state, or of another lattice, boundaries, precision or engine;
 *     PFL_ERR_STATE for a state with solid cells loaded into a context created
 *     without solids (or the reverse).
 * Both synchronise the stream. */
size_t pfl_state_bytes(const pfl_ctx* ctx);
pfl_status pfl_save(pfl_ctx* ctx, void* buf, size_t bytes);
pfl_status pfl_load(pfl_ctx* ctx, const void* buf, size_t bytes);

/* FP64 reductions over the domain (section "Rising bubble": centre of mass):
 *   out[0] = sum phi, out[1..3] = sum phi * (x, y, z),
 *   out[4] = sum (1 - phi), out[5..7] = sum (1 - phi) * (x, y, z).
 * nonfinite (may be NULL) receives the number of cells whose phi is NaN/Inf.
 * Returns PFL_ERR_UNSTABLE when that number is non-zero or when the largest
 * flow speed |u| over the fluid cells (pfl_max_speed) exceeds
 * PFL_SPEED_LIMIT; out and nonfinite are filled in either case.
 * Synchronises. */
pfl_status pfl_diag(pfl_ctx* ctx, double out[8], long long* nonfinite);

/* Largest flow speed max |u| over the fluid cells of the current state, with
 * u = sum_i c_i g_i + F / (2 rho) as in pfl_fields; a NaN/Inf velocity gives
 * +inf.  umax: one double, host or device.  Synchronises. */
pfl_status pfl_max_speed(pfl_ctx* ctx, double* umax);

/* Interface height of the column (x, z) (the amplitude measure of the wave
 * cases, section "Gravity wave", "Capillary wave"): the first j, going up
 * along y, with phi_j >= 1/2 > phi_{j+1}, interpolated linearly:
 * y = j + (phi_j - 1/2) / (phi_j - phi_{j+1}), in FP64 from the stored phi.
 * NaN when the column has no such crossing.  y: one double, host or device.
 * PFL_ERR_ARG for a column outside the lattice.  Synchronises. */
pfl_status pfl_interface_height(pfl_ctx* ctx, int x, int z, double* y);

/* Advance n_steps > 0 steps like pfl_step, recording a CUDA event pair on the
 * context's stream around every kernel launch; ms[0] receives the summed
 * device time of the stream-collide kernel, ms[1] that of the phi pass
 * (section "The lattice Boltzmann method": the fused collide-stream, then
 * phi = sum h).  Measurement aid; synchronises. */
pfl_status pfl_kernel_times(pfl_ctx* ctx, int n_steps, double ms[2]);

/* Device bytes of the adjoint workspace for an adjoint over n_steps steps
 * (0 if ctx is NULL or n_steps < 1).  It holds ceil(n_steps / K) checkpoints
 * and K recomputed states with K = ceil(sqrt(n_steps)), two adjoint
 * population sets, the observation weights and the reduction scratch. */
size_t pfl_adjoint_workspace_bytes(const pfl_ctx* ctx, int n_steps);

/* Discrete adjoint of n_steps time steps from the current state: the gradient
 * of J = sum_o sum_x W_o(x) phi(x, t0 + s_o) with respect to the mobility M,
 * the interface width xi and the surface tension sigma -- the parameters the
 * paper finds the PFLBM's accuracy sensitive to (sections "Rising bubble",
 * mobility study).  Bubble rise velocity (the centroid of 1 - phi, linear in
 * phi because sum(1 - phi) is conserved) and the amplitude of a wave mode are
 * such functionals.
 *   obs_steps: n_obs distinct steps in [0, n_steps], relative to the current
 *   time; obs_weights: n_obs arrays of N doubles (host or device; device
 *   arrays are read in place, host arrays copied in when their step comes).
 *   A nonlinear J of phi at those steps is differentiated by passing the
 *   weights W_o = dJ / dphi(t_o) evaluated on a forward run (chain rule):
 *   the gradient returned is then dJ / d(M, xi, sigma), while *J holds the
 *   linear functional sum_o W_o . phi(t_o) of those weights.
 *   The forward run keeps a checkpoint every K = ceil(sqrt(n_steps)) steps,
 *   and the reverse sweep recomputes one K-step segment at a time.
 *   On return the context holds the state after n_steps steps (as pfl_step);
 *   *J receives J, grad[0..2] = dJ/dM, dJ/dxi, dJ/dsigma: the exact
 *   derivative of the discrete map.  Over horizons on which the flow amplifies
 *   perturbations it grows far beyond any finite-difference estimate (the
 *   128x384x128 bubble: within 1e-3 of central differences at 2000 steps,
 *   50-2400x them at 4000, where the differences themselves stop converging).
 *   adj_workspace: device memory of pfl_adjoint_workspace_bytes() bytes,
 *   256-byte aligned, caller-owned.
 * PFL_ERR_STATE for FP16S storage, the BGK mode or lattices with 27 N >= 2^32;
 * PFL_ERR_ARG for bad observations (NULL weights, steps outside [0, n_steps]
 * or repeated).  Synchronises. */
pfl_status pfl_adjoint(pfl_ctx* ctx, int n_steps, int n_obs, const int* obs_steps, const double* const* obs_weights,
                       void* adj_workspace, size_t adj_bytes, double* J, double grad[3]);

/* ------------------------------------------------------------------ batch --
 * Many independent lattices of uneven size, each with its own parameters
 * (M, xi, sigma, densities, ...), advanced together: every lattice step is
 * one persistent grid-stride launch of the fused two-array step per class of
 * instances (one z plane, and 3-D) over a work list of (instance, xy tile,
 * z chunk) tiles -- the single-lattice step's tile code, phi formed in the
 * step -- and pfl_batch_step replays a CUDA graph of 16 steps.  Each instance
 * evolves bitwise as the same lattice run alone with the fused engine.  All instances share the precision (FP64 or
 * FP32); MRT and the D3Q15 phase field only; 27 N < 2^32 per instance. */
typedef struct pfl_batch pfl_batch;

/* Device bytes of the batch workspace (0 if a parameter set is invalid,
 * precisions differ or are FP16S, the collision is not MRT or the h lattice
 * is D3Q27). */
size_t pfl_batch_workspace_bytes(const pfl_params* params, int count);

/* Create the batch: params[count]; phi0[count] arrays (host or device, N_i
 * doubles each, required); u0, p0: NULL or arrays of count pointers (entries
 * may be NULL).  tune_shapes != 0 times the candidate launch shapes of each
 * class on the initial state and keeps the fastest -- tile height 4 or 8
 * (128 or 256 threads per block) for one z plane, the z chunk (a cost
 * model's, 8, 16, 32, whole) in 3-D, grid 1, 2 or 4 x SMs x resident blocks
 * -- then rebuilds the initial state.  Without tuning: tile height 4 / 8, the
 * cost model's z chunk, grid SMs x resident blocks.  Synchronises. */
pfl_status pfl_batch_init(const pfl_params* params, int count, const double* const* phi0, const double* const* u0,
                          const double* const* p0, void* workspace, size_t workspace_bytes, void* stream,
                          int tune_shapes, pfl_batch** out);

/* Advance every active instance n_steps steps (asynchronous). */
pfl_status pfl_batch_step(pfl_batch* b, int n_steps);

/* Fields of instance i, as pfl_fields.  Synchronises. */
pfl_status pfl_batch_fields(pfl_batch* b, int i, double* phi, double* rho, double* p, double* u);

/* pfl_diag of every instance: out[8 * count] (may be NULL), nonfinite[count]
 * (may be NULL).  Instances whose phi holds NaN/Inf or whose flow speed
 * exceeds PFL_SPEED_LIMIT are stopped (skipped by later steps, their state
 * kept) and the call returns PFL_ERR_UNSTABLE.  Synchronises. */
pfl_status pfl_batch_diag(pfl_batch* b, double* out, long long* nonfinite);

/* Launch shape of class cls (0: one z plane, 1: 3-D), in place of the one
 * the tuner or the default chose: tiles of tile_x x tile_y cells, one block of
 * tile_x x tile_y threads each (class 0: 32x4, 32x8, and in FP32 16x8; class
 * 1: 32x8, 16x8, and in FP32 16x16); z_chunk planes per tile (class 1; 0: the
 * whole lattice); grid blocks of the persistent launch (0: SMs x resident
 * blocks; capped by the tile count).  Rebuilds the class's work list and the
 * CUDA graph; results do not depend on the shape (every cell's arithmetic is
 * the same).  PFL_ERR_ARG for a shape the class and precision do not have.
 * Synchronises. */
pfl_status pfl_batch_set_shape(pfl_batch* b, int cls, int tile_x, int tile_y, int z_chunk, int grid);

/* Launch shape chosen for each of the two classes (0: one z plane, 1: 3-D):
 * threads per block, grid blocks and work-list tiles (each array of 2, may be
 * NULL). */
pfl_status pfl_batch_shapes(const pfl_batch* b, int* threads, int* grid, int* ntiles);

/* Steps taken by the batch (-1 for NULL). */
long long pfl_batch_time(const pfl_batch* b);

/* Release the batch (the caller frees the workspace afterwards). */
void pfl_batch_destroy(pfl_batch* b);

/* Mass and centre-of-mass sums of a phase field the caller already holds,
 * computed without any device memory from the caller: for callers that are
 * not allowed to allocate device memory themselves -- an application whose
 * GPU memory all belongs to its own pool or caching allocator, a plugin given
 * fixed buffers and no right to allocate, a loop that cannot pay for the
 * device synchronisation an allocation may cause.  The paper has no
 * counterpart; this is a service of the library.
 *   phi: device pointer to nx*ny*nz values, x-fastest; FP64 if phi_fp64 != 0,
 *        else FP32 (the caller keeps ownership).
 *   out: host array of 8 doubles, the same sums as pfl_diag; nonfinite (host,
 *        may be NULL) the number of NaN/Inf values.  stream: a cudaStream_t.
 * Scratch: a fixed array inside the library image (about 88 KB per device,
 * held until the process exits); no cudaMalloc/cudaFree is called.  Every
 * call looks up that array's device address on phi's device, so a device
 * whose context was reset is picked up by the next call; the first call on a
 * device also loads the library's kernels there, so make it before any stream
 * capture.  The kernels run on phi's device; the caller's current device is
 * the same after the call as before it.  All calls on one device share the
 * array: calls that overlap on the GPU race and must be ordered by the
 * caller.
 * Errors: PFL_ERR_ARG for NULL pointers, non-device phi, dims < 1 or more than
 * 2^31 - 1 cells; PFL_ERR_UNSTABLE when NaN/Inf are present; PFL_ERR_CUDA.
 * Synchronises the stream. */
pfl_status pfl_phi_moments_static(const void* phi, int phi_fp64, int nx, int ny, int nz, double out[8],
                                  long long* nonfinite, void* stream);

/* Time steps taken since pfl_init (or -1 for a NULL context). */
long long pfl_time(const pfl_ctx* ctx);

/* Release the host context (the caller frees the workspace afterwards). */
void pfl_destroy(pfl_ctx* ctx);

/* Message of the last failed call on this thread ("" if none). */
const char* pfl_last_error(void);

/* Library interface version (2: pfl_params carries hydrostatic and p_level;
 * 3: pfl_hydrostatic_pstar). */
int pfl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PFLBM_H */
