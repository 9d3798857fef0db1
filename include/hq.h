/*
 * hq.h -- C ABI of a GB300 (sm_103a) implementation of the quasi-static PIC
 * per-slice loop of arXiv:2109.10277 (HiPACE++), Sec. 2 and Sec. 3.
 *
 * Units are the paper's normalized units (Sec. 6, "normalized units"): lengths
 * in 1/k_p, fields in E0 = m c omega_p / e, densities in n0, c = eps0 = mu0 = 1.
 * The default plasma is electrons (charge -1, mass 1) over immobile ions; hq_grid_desc.species
 * gives plasmas of several species with their own charge and mass (mobile ions).
 *
 * Conventions for every entry point:
 *  - Pointers named "device" must point to CUDA device memory (for example the
 *    data of a torch CUDA tensor); the caller owns them and keeps them alive
 *    until the work queued on the grid's stream has finished.
 *  - Calls are asynchronous on the stream given to hq_grid_create.  Argument and
 *    ordering errors are reported synchronously by the return value; faults seen
 *    inside kernels (a bounded wait that ran out, a non-finite field) set a device
 *    status word that hq_sync reports.
 *  - No C++ exception crosses this boundary.  After a non-OK status,
 *    hq_last_error(grid) returns a message (valid until the next call on the grid).
 *  - A grid is used by one host thread at a time.
 *
 * Data layout: a transverse field slice is ny x nx values, row-major, row = y.
 * Node (iy, ix) sits at (xmin + ix*dx, ymin + iy*dy); nodes 0 and nx (ny) lie on
 * the Dirichlet wall, so row 0 and column 0 of every field are zero.  Field
 * values are double for HQ_PREC_FP64 grids and float for the FP32 precisions.
 * Beam arrays are always double.
 *
 * Run-time switches (environment variables, read when a grid is created; HQ_NO_GRAPH
 * at every hq_sweep_step, HQ_NO_FORK whenever a sweep is issued or captured, not when a
 * captured one is replayed); each turns an optimization off and leaves the results
 * unchanged up to summation order:
 *   HQ_NO_FOLD=1   FP32 DST-I without the folded (half-K) products
 *   HQ_SOLVE_BN=64 FP32 solves always on 128 x 64 tiles (no 128 x 32 tiles)
 *   HQ_NO_RS=1     FP32 square grids of 256 or 512 cells: the solve streams the fold matrix
 *                  per tile instead of keeping each CTA's slice of it in shared memory
 *   HQ_NO_PDL=1    no programmatic dependent launch between the per-slice kernels
 *   HQ_NO_GRAPH=1  hq_sweep_step issues its launches instead of replaying a CUDA graph
 *   HQ_NO_FORK=1   hq_sweep_step keeps the witness sums and beam deposits on the grid's
 *                  stream instead of beside the final pass on a second stream
 *   HQ_SEPARATE_SRC=1  FP32: the psi/Ez/Bz and B_perp sources are formed by kernels of
 *                  their own ahead of each solve instead of in the solve's first phase
 *   HQ_NO_F4CACHE=1  FP32: every predictor-corrector trial pass and the final pass gather all
 *                  six fields (by default the first trial pass of a slice keeps ExmBy, EypBx,
 *                  Ez, Bz per particle and the later passes of the slice gather Bx, By alone;
 *                  the gathered values are bit for bit the same)
 *   HQ_NO_SRCCACHE=1  FP32: every B_perp source phase of the predictor-corrector forms all its
 *                  terms from the records (by default the first iteration of a slice keeps
 *                  the part that does not depend on the trial J_perp, and the others add the
 *                  trial term to it: the same sources up to FP32 rounding)
 * and one switch for testing the failure path, which does change results:
 *   HQ_FAULT_BARRIER=1  (FP32 grids) the first grid barrier of every tensor-core solve
 *                  waits for one CTA more than the launch has, so its bounded wait runs
 *                  out after about two seconds; the solve returns early with an
 *                  incomplete result and hq_sync reports HQ_ERR_TIMEOUT
 */
#ifndef HQ_H
#define HQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HQ_OK = 0,
  HQ_ERR_ARG = 1,      /* invalid argument (null pointer, size out of range)          */
  HQ_ERR_CUDA = 2,     /* a CUDA runtime call failed                                   */
  HQ_ERR_OOM = 3,      /* a device allocation failed                                   */
  HQ_ERR_NUMERIC = 4,  /* a non-finite value reached the field solve                  */
  HQ_ERR_TIMEOUT = 5,  /* a bounded device-side wait ran out (kernel returned early)   */
  HQ_ERR_STATE = 6,    /* call out of order (slices must be visited 0, 1, 2, ...)      */
  HQ_ERR_UNSUPPORTED = 7
} hq_status;

typedef enum {
  /* everything in FP64, DST-I by an FP64 FFT */
  HQ_PREC_FP64 = 0,
  /* push/gather/deposit in FP32 with FP64 position and Psi accumulators; the DST-I
     as dense products on the tensor cores with each FP32 operand split into two
     bf16 terms (3 products, FP32 accumulation) */
  HQ_PREC_FP32_BF16X3 = 1,
  /* the same FP32 path with each DST operand split into two TF32 terms instead (hi = the value
     rounded to TF32, lo = the remainder, read by the tensor core truncated to TF32): ~21
     significant bits per operand against bf16x3's 16, at twice the operand bytes and twice
     the tensor-core instructions (K = 8 per instruction); every grid shape takes the solve
     that streams the sine/fold matrices (the resident-matrix solve would need 256 KB of
     shared memory at 512^2) */
  HQ_PREC_FP32_TF32X3 = 2
} hq_precision;

/* One plasma species (Sec. 6: plasmas of several species and profiles, ion motion).  The
 * push takes the species' q/M (Sec. 3.2 plasma equations), the deposits q (and q^2/M for chi).
 * Placement as for the default plasma: ppc_x x ppc_y particles per cell at sub-cell centres,
 * weight n0_scale * n(r) * dx * dy / ppc.  neutralize = 1: an immobile background of the
 * opposite charge sits at the species' initial positions (the default electrons' ions); 0:
 * the species' own initial charge stays in the slice (e.g. electrons and mobile ions placed
 * alike neutralize each other). */
typedef struct {
  double charge, mass;              /* units of e and m_e: the default electrons are -1, 1 */
  double n0_scale;
  int32_t ppc_x, ppc_y;             /* 1..16 each                                          */
  const double* radial_profile;     /* host; n_profile entries over [0, profile_rmax]; NULL = uniform */
  int32_t n_profile;
  double profile_rmax;
  int32_t neutralize;               /* 0 or 1                                               */
} hq_species_desc;

/* Grid, plasma and solver description; every field is copied by hq_grid_create.
 * Sec. 2 (slice loop), Sec. 3.2 (push, deposition, Poisson and P-C solvers). */
typedef struct {
  int32_t nx, ny, nzeta;            /* cells; 8 <= nx, ny <= 4096, nzeta >= 1          */
  double xmin, xmax, ymin, ymax;    /* Dirichlet box                                   */
  double zeta_min, zeta_max;        /* slice i covers zeta_max - (i+1) dz .. - i dz    */
  int32_t shape_order;              /* transverse B-spline order 0..3 (Sec. 3.2)       */
  int32_t ppc_x, ppc_y;             /* plasma particles per cell, at sub-cell centres  */
  const double* radial_profile;     /* host; n_profile entries over r in [0, rmax],
                                       linearly interpolated; NULL = uniform           */
  int32_t n_profile;
  double profile_rmax;
  double n0_scale;                  /* multiplies plasma (and ion) density            */
  int32_t n_pc_iter;                /* predictor-corrector iterations, or the explicit
                                       solver's conjugate-gradient iterations (fixed count) */
  double pc_mix;                    /* B <- pc_mix * B_solved + (1 - pc_mix) * B      */
  double psi_guard;                 /* particle removed when 1 + Psi < psi_guard      */
  int32_t precision;                /* hq_precision                                   */
  int32_t bperp_solver;             /* hq_bperp_solver (0: predictor-corrector)       */
  int32_t resort_every;             /* m > 0: after the final push to slice i with i % m
                                       == 0 the plasma slice is re-sorted by cell (stable
                                       counting sort, Sec. 3.1); 0: never.  Refused by
                                       hq_sweep_forward_ckpt (HQ_ERR_UNSUPPORTED)          */
  int32_t deterministic;            /* 1 (FP64 precision): every plasma and beam deposit
                                       (with the explicit solver also its source deposits and
                                       dot products, summed in a fixed order) and the witness sums
                                       accumulate in 64-bit fixed point (resolution 2^-72,
                                       contributions and sums below 2^31 in magnitude, else
                                       HQ_ERR_NUMERIC) with integer atomics, so a sweep's
                                       results do not depend on the order of the atomic
                                       additions: bitwise reproducible.  Refused by
                                       hq_sweep_forward_ckpt (HQ_ERR_UNSUPPORTED); 0: FP64
                                       atomics (last-bit run-to-run differences)          */
  const hq_species_desc* species;   /* host array of n_species (1..4) plasma species, copied;
                                       the plasma slice holds them one after the other
                                       (species s from sum_{t<s} nx ny ppc_t on); with
                                       species the grid's ppc_x, ppc_y, radial_profile,
                                       profile_rmax and n0_scale do not place the plasma.
                                       Not with the re-sort or the checkpointed forward
                                       (HQ_ERR_UNSUPPORTED); the explicit solver's
                                       preconditioner shift is then sum q^2 n0_scale / M  */
  int32_t n_species;                /* 0: the default electrons (q = -1, M = 1) over
                                       immobile ions, placed by the fields above          */
  int32_t pc_residuals;             /* 1: record the predictor-corrector residual of every
                                       slice for hq_pc_residuals (the last iteration's
                                       solve launch sums it: ~6 us more per slice); 0: off */
} hq_grid_desc;

/* B_perp field solver (Sec. 3.2: "predictor-corrector field solver" and "explicit field
 * solver").  The explicit solver differentiates the deposited plasma current along zeta
 * with the particle equations (a reading: the paper cites the equation), which turns
 * Eq. bxby into (L - chi) Bx = -dy Jz + Ty, (L - chi) By = dx Jz - Tx with chi =
 * sum q^2 w S / (M (1+Psi) A) and T the B-independent part of d(J_perp)/d(zeta) (plasma:
 * deposited force and convective terms; beams: central differences of their slice
 * deposits); it is solved by n_pc_iter preconditioned conjugate-gradient iterations
 * (preconditioner (c - L)^{-1} with c the unperturbed chi: n0_scale, or sum q^2 n0_scale / M
 * over the plasma species; one shifted DST-I solve each) from the guess 2 B(i-1) - B(i-2).
 * The adjoint supports only the predictor-corrector. */
typedef enum { HQ_BPERP_PC = 0, HQ_BPERP_EXPLICIT = 1 } hq_bperp_solver;

/* One beam species, structure of arrays in DEVICE memory (double), n particles.
 * x, y, zeta and ux, uy, uz (normalized momenta) are updated in place by the
 * beam push; w is the number of physical particles per macroparticle in units
 * of n0 / k_p^3. */
typedef struct {
  int64_t n;
  double *x, *y, *zeta, *ux, *uy, *uz, *w;
  double charge, mass;              /* units of e and m_e                              */
} hq_beam_view;

/* Per-slice field outputs, DEVICE arrays of nzeta x ny x nx elements of the grid's
 * field type (see top); a NULL member is not written.  rho and J are totals
 * (plasma + ions + beams); exmby = Ex - By, eypbx = Ey + Bx (Eq. exmby). */
typedef struct {
  void *rho, *jx, *jy, *jz, *chi, *psi, *exmby, *eypbx, *ez, *bx, *by, *bz;
} hq_field_out;

/* Read-only DEVICE views of the plasma slice (library-owned memory, valid until
 * hq_grid_destroy).  x, y, psi are double; ux, uy, w are of the field type;
 * alive is uint8 (0 once a particle is removed).  origin (int32) gives each entry's
 * index in the initial placement (cell-row-major, ppc_x x ppc_y sub-cells per cell) when
 * the grid re-sorts its plasma (resort_every > 0); NULL otherwise, when entry p is
 * particle p of that placement. */
typedef struct {
  int64_t n;
  const double *x, *y, *psi;
  const void *ux, *uy, *w;
  const uint8_t* alive;
  const int32_t* origin;
} hq_plasma_view;

typedef struct hq_grid_s* hq_grid_t;

/* Creates a grid: validates desc, allocates the plasma slice, field slices and
 * transform scratch on the current device, and builds the DST tables.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: HQ_ERR_ARG (bad desc), HQ_ERR_OOM, HQ_ERR_CUDA, HQ_ERR_UNSUPPORTED
 * (the FP32 precisions need a compute capability 10.x device). */
hq_status hq_grid_create(const hq_grid_desc* desc, void* cuda_stream, hq_grid_t* out);

/* Frees everything the grid owns (synchronizes its stream first). NULL is a no-op. */
hq_status hq_grid_destroy(hq_grid_t grid);

/* Sec. 2 step 1-2: for slice 0, resets the plasma to its unperturbed state ahead of
 * the beams (Sec. 2, "a slice of unperturbed plasma is initialized ahead of the
 * beams") and deposits it.  For slice i > 0, gathers the converged fields of slice
 * i-1, takes the final AB5 step (Sec. 3.2 plasma push) to slice i, applies the
 * removal rule, and deposits rho, J, chi of slice i.  Requires hq_solve_fields(i-1)
 * (HQ_ERR_STATE otherwise). */
hq_status hq_advance_slice(hq_grid_t grid, int32_t slice);

/* Sec. 2 step 3 and Sec. 3.1 (beams sorted per slice): adds the charge and
 * current of the beam particles whose zeta falls in slice i (order 0
 * longitudinally), and stores J_perp of slice i+1 for the predictor-corrector.
 * Views are binned by slice (counting sort on the device on their current zeta): on
 * slice 0 all of them; on a later slice only a view not passed at the slice before
 * (its particles must not have been pushed in this sweep), while a view passed before
 * keeps its bins and a view no longer passed is forgotten.  So a beam can arrive box
 * by box (Sec. 5.2 temporal pipeline): pass the next box's view on the last slice of
 * the current one, whose J_perp(i+1) it supplies.  At most 4 views per call.  Requires
 * hq_advance_slice(i). */
hq_status hq_beam_deposit(hq_grid_t grid, const hq_beam_view* beams, int32_t nbeams, int32_t slice);

/* Sec. 2 steps 4-7 and Sec. 3.2 (fast Poisson solver, predictor-corrector):
 * solves psi and ExmBy, EypBx = -grad psi (Eq. psi, exmby), Ez (Eq. ez), Bz (Eq. bz),
 * then n_pc_iter predictor-corrector iterations for Bx, By (Eq. bxby).
 * Requires hq_beam_deposit(i) (nbeams may be 0). */
hq_status hq_solve_fields(hq_grid_t grid, int32_t slice);

/* Copies the fields of the last solved slice into out at element offset
 * slot * ny * nx (Sec. 3.1: per-slice diagnostics). */
hq_status hq_store_fields(hq_grid_t grid, const hq_field_out* out, int64_t slot);

/* Sec. 3.2 (beam pusher): advances the particles of slice i of each beam by dt
 * with a second-order drift-kick-drift step (Boris kick) in the fields of the last
 * solved slice, which must be i.  Positions and momenta are updated in place.  Each
 * view must have been passed to hq_beam_deposit(i) (HQ_ERR_STATE otherwise). */
hq_status hq_push_beams(hq_grid_t grid, hq_beam_view* beams, int32_t nbeams, int32_t slice, double dt);

/* Adds sum(q w), sum(q w Ez), sum(q w Ez^2) over the particles of slice i of
 * `beam` (Ez gathered with the grid's shape) to sums[0..2] (DEVICE double[3]). */
hq_status hq_witness_accumulate(hq_grid_t grid, const hq_beam_view* beam, int32_t slice, double* sums);

/* Sec. 3.2 (predictor-corrector): the relative change of B_perp in the last iteration of each
 * slice of the last sweep, ||B_m - B_m-1|| / ||B_m|| over both components and every node (the
 * mixing's own residual; 0 for a slice with no iteration, or with the explicit solver, which has
 * no mixing), written to out[0..n) (HOST doubles; entries past nzeta are 0).  Recorded only by a
 * grid created with pc_residuals = 1 (HQ_ERR_STATE otherwise).  Synchronizes the grid's stream.
 * Errors: HQ_ERR_ARG, HQ_ERR_STATE. */
hq_status hq_pc_residuals(hq_grid_t grid, double* out, int32_t n);

/* Sec. 3.1 (beam particles sorted per slice) and Sec. 5.2 (temporal pipeline: a box's
 * particles are handed to the next time step): writes the slice of every particle of
 * `beam` to slices[0..n) (DEVICE int32[n]) with the arithmetic hq_beam_deposit bins by,
 * floor((zeta_max - zeta) / dzeta) in FP64: 0..nzeta-1 inside the box, -1 ahead of its
 * head (zeta above zeta_max), nzeta behind its tail, -2 for a non-finite zeta.  Queued on
 * the grid's stream; needs no slice state.  Errors: HQ_ERR_ARG. */
hq_status hq_beam_slices(hq_grid_t grid, const hq_beam_view* beam, int32_t* slices);

/* Sec. 6 (precision study: the witness beam's emittance over many time steps): adds the
 * weighted raw moments of all particles of `beam` to moments[0..10] (DEVICE double[11],
 * zeroed by the caller): sum w, sum w x, sum w y, sum w ux, sum w uy, sum w x^2, sum w y^2,
 * sum w ux^2, sum w uy^2, sum w x ux, sum w y uy (FP64).  The normalised rms emittance
 * follows as eps_x^2 = <x^2><ux^2> - <x ux>^2 with centred, weight-averaged moments.
 * Queued on the grid's stream; the beam needs no binning.  Errors: HQ_ERR_ARG. */
hq_status hq_beam_moments(hq_grid_t grid, const hq_beam_view* beam, double* moments);

/* One full quasi-static sweep head -> tail (Sec. 2, Fig. 1): for every slice,
 * advance, beam deposit, field solve, then optionally store the fields (out may be
 * NULL), push the beams (dt != 0), and accumulate witness sums (witness_beam >= 0,
 * witness_sums a DEVICE double[3], zeroed by the caller).  After the last slice the
 * plasma is advanced once more, so hq_plasma_state shows the state past the box. */
hq_status hq_sweep_step(hq_grid_t grid, hq_beam_view* beams, int32_t nbeams, double dt,
                        const hq_field_out* out, int32_t witness_beam, double* witness_sums);

/* Slices [slice_begin, slice_end) of a sweep: per slice the steps of hq_sweep_step (advance, beam
 * deposit, solve, optional store / witness sums / push) with the views `beams`; on the range's
 * last slice the views `next` (nnext of them; may be NULL with nnext = 0) join the beam
 * deposit, so that the J_perp of slice slice_end reaches the predictor-corrector.  This is one
 * box of the Sec. 5.2 temporal pipeline: the box's particles in `beams`, the next box's in
 * `next` (pass them for the box's last slice only, in a call of its own, to receive them as
 * late as possible).  slice_begin must be 0 (a new sweep) or the previous call's slice_end;
 * slice_end <= nzeta, nbeams + nnext <= 4; reaching nzeta advances the plasma once more as
 * hq_sweep_step does.  Launched from the host slice by slice (no graph replay).  Errors:
 * HQ_ERR_ARG, HQ_ERR_STATE (out of order), and those of the per-slice calls. */
hq_status hq_sweep_slices(hq_grid_t grid, hq_beam_view* beams, int32_t nbeams, const hq_beam_view* next,
                          int32_t nnext, int32_t slice_begin, int32_t slice_end, double dt,
                          const hq_field_out* out, int32_t witness_beam, double* witness_sums);

/* Forward sweep for differentiation (gradients are a goal the paper names, Sec. 1, with
 * no adjoint formulation): the same sweep as hq_sweep_step with dt = 0 and no field output, but
 * it stores a checkpoint (plasma slice with its AB5 history and the field records a
 * slice starts from) every ckpt_every slices, and the per-slice tapes of the last
 * segment.  witness_sums (DEVICE double[3], zeroed by the caller) receives
 * sum q w (1, Ez, Ez^2) over witness_beam (-1: none).  Memory: about
 * (nzeta/ckpt_every) checkpoints + ckpt_every tapes, each ~(P x 130 B + n^2 x 80 B)
 * in FP32; HQ_ERR_OOM asks for a larger or smaller interval. */
hq_status hq_sweep_forward_ckpt(hq_grid_t grid, hq_beam_view* beams, int32_t nbeams, int32_t witness_beam,
                                double* witness_sums, int32_t ckpt_every);

/* Reverse-zeta adjoint of the last hq_sweep_forward_ckpt (same beams and witness):
 * given dL/d(S0, S1, S2) of the witness sums (HOST double[3]; may be NULL without a
 * witness) and, optionally, the adjoint seeds of per-slice output fields (dL_dfields:
 * DEVICE arrays of nzeta x ny x nx field-type values holding dL/d(field) per slice and
 * node, NULL members and a NULL struct meaning zero; rho, jx, jy, jz, psi, exmby, eypbx,
 * ez, bx, by, bz are supported, chi is refused with HQ_ERR_ARG; seeds on wall nodes are
 * ignored, the forward holds those fields at zero), returns dL/dw for
 * every beam particle (dL_dbeam_w: HOST array of nbeams DEVICE double* of n entries,
 * overwritten; an entry may be NULL), dL/dw of every plasma particle (DEVICE double[P],
 * may be NULL), dL/dn0_scale (DEVICE double[1], may be NULL) and dL/d(radial profile)
 * (DEVICE double[n_profile], may be NULL).  Segments are recomputed from their
 * checkpoints; deposit and gather are transposes of each other, the DST-I solve is
 * self-adjoint, central differences transpose to minus themselves, and the push has
 * its own adjoint kernel.  Leaves the grid's forward state undefined (the next sweep
 * restarts at slice 0).  Errors: HQ_ERR_STATE without a matching forward. */
hq_status hq_sweep_adjoint(hq_grid_t grid, hq_beam_view* beams, int32_t nbeams, int32_t witness_beam,
                           const double* dL_dsums, const hq_field_out* dL_dfields, double* const* dL_dbeam_w,
                           double* dL_dplasma_w, double* dL_dn0_scale, double* dL_dprofile);

/* Solves nrhs (1..5) Dirichlet Poisson problems L f = s with the grid's DST-I
 * backend (Sec. 3.2, fast Poisson solver): src and dst are DEVICE arrays of
 * nrhs x ny x nx field-type values (row/col 0 of src are ignored). */
hq_status hq_poisson_solve(hq_grid_t grid, const void* src, void* dst, int32_t nrhs);

/* Allocation-free Dirichlet Poisson solve.  The paper has no counterpart: this is
 * an addition for callers that cannot allocate device memory.  Such callers
 * exist: a host application that reserved the whole device memory pool up front
 * and lets no library allocate from it, code in a latency-critical loop where a
 * cudaMalloc or cudaFree would stall or synchronize the device, and code that is
 * not allowed to create device objects after start-up.  This entry point solves
 * the same problem as hq_poisson_solve on an FP32 (bf16x3 tensor-core DST-I) grid
 * but needs no grid object and allocates nothing: its scratch is one fixed,
 * file-scope static device array of 9 MiB + 256 bytes, which every GPU that loads
 * libhq holds until the process exits.
 *
 * src, dst: DEVICE float arrays of nrhs x ny x nx, row-major, row = y (row and
 * column 0 of src are ignored; dst has zeros there).  dx, dy: node spacings.
 * Limits set by the static array: 8 <= nx, ny <= 512 and 1 <= nrhs <= 3; anything
 * larger returns HQ_ERR_ARG with a message naming the limit.
 * cuda_stream: the cudaStream_t the work is queued on (NULL = legacy stream).
 * The first call on each device does that device's set-up (it looks up the static
 * array's device address and raises the GEMM's shared-memory limit); make that
 * first call before any stream capture.  A call with a new (nx, ny, dx, dy)
 * rebuilds the sine and 1/lambda tables inside the array.  Every call shares the
 * one array, which keeps the last call's contents: calls whose work overlaps on
 * the GPU (several streams, several host threads) race, so the caller must
 * serialize them.  A call made while its stream is being captured always enqueues
 * the table build, and the next call rebuilds the tables again.  cuda_stream must
 * belong to the current device.  The call is asynchronous: a bounded device wait
 * that ran out (incomplete result) or a non-finite result is flagged in a status
 * word at the start of the array, which stays set until hq_sync(NULL, ...) reports
 * and clears it.  Errors returned directly: HQ_ERR_ARG, HQ_ERR_CUDA,
 * HQ_ERR_UNSUPPORTED (not an sm_103a device); the message is read with
 * hq_last_error(NULL). */
hq_status hq_poisson_solve_static(const float* src, float* dst, int32_t nx, int32_t ny, double dx, double dy,
                                  int32_t nrhs, void* cuda_stream);

/* Fills *out with views of the plasma slice (state after the last advance). */
hq_status hq_plasma_state(hq_grid_t grid, hq_plasma_view* out);

/* Kernel classes timed by the profiler (index into hq_profile_t arrays). */
enum {
  HQ_K_FINAL = 0,   /* plasma final pass: gather, AB5 step, deposit (Sec. 3.2)        */
  HQ_K_TRIAL = 1,   /* plasma predictor-corrector trial pass                           */
  HQ_K_DST = 2,     /* DST-I transform launches (tensor-core GEMM or FP64 FFT)         */
  HQ_K_FIELD = 3,   /* source assembly, -grad psi, mixing, guess/shift, output copy    */
  HQ_K_BEAM = 4,    /* beam binning, deposit, push, witness sums                       */
  HQ_K_OTHER = 5,   /* buffer resets, plasma initialization                            */
  HQ_K_CLASSES = 8
};
typedef struct {
  double ms[HQ_K_CLASSES];        /* summed device time (CUDA events on the grid's stream) */
  int64_t launches[HQ_K_CLASSES]; /* kernel launches issued                                 */
} hq_profile_t;

/* on != 0: from now on record a CUDA event pair around every kernel-class launch
 * group on the grid's stream; on == 0: stop recording.  Launch counting is always
 * on.  Either call resets the accumulators. */
hq_status hq_profile_enable(hq_grid_t grid, int32_t on);

/* Synchronizes the stream and returns the accumulated times and launch counts. */
hq_status hq_profile_read(hq_grid_t grid, hq_profile_t* out);

/* Waits for the grid's stream, then reports device status: HQ_ERR_TIMEOUT or
 * HQ_ERR_NUMERIC if a kernel flagged one (the flag is cleared), else HQ_OK.
 * removed (may be NULL) receives the number of plasma particles removed so far.
 * grid == NULL: waits for all work on the current device (cudaDeviceSynchronize) and
 * reports the status of the hq_poisson_solve_static calls made on it since the last
 * such query: HQ_ERR_TIMEOUT if a bounded wait inside one ran out (its result is
 * then incomplete), HQ_ERR_NUMERIC if one produced a non-finite value, else HQ_OK;
 * the flag is cleared and *removed (if given) is set to 0.  Allocates nothing.
 * HQ_ERR_CUDA if the device cannot be synchronized (e.g. there is none). */
hq_status hq_sync(hq_grid_t grid, int64_t* removed);

/* Message for the last non-OK status on this grid (or a global message when
 * grid is NULL, e.g. after a failed hq_grid_create). */
const char* hq_last_error(hq_grid_t grid);

#ifdef __cplusplus
}
#endif
#endif /* HQ_H */
