/*
 * vofp.h -- C ABI of libvofp, a single-GPU (sm_103a) solver for the pressure-projection Poisson
 * equation of the cartesian-grid volume-of-fluid method of Dommermuth et al., "The numerical
 * simulation of ship waves using cartesian-grid and volume-of-fluid methods".
 *
 * The equation (Sec. 2 Eq. pois; Sec. 2.1 Eq. poisson1) is  div( grad(p) / rho ) = div(u*) / dt,
 * integrated over each cell's open faces (Sec. 2.3 Eqs. integral1-integral2).  The library solves
 * the discrete form  A_hat p = b_hat  where
 *   - A_hat = P^T A P is symmetric positive (semi)definite: A is the 7-point finite-volume operator
 *     with face coefficients T_f = A_f S_f / ((d_L rho_L + d_R rho_R) / 2) (aperture x face area x
 *     half-cell harmonic average of 1/rho over centre distance), and P merges cells whose open
 *     volume is below a threshold into a neighbour (Sec. 2.3);
 *   - b = -(1/dt) * (sum of outward face fluxes A_f S_f u_f + body-surface flux), Sec. 2.4 F_i;
 *   - rho = rho_gas + (rho_liquid - rho_gas) F from the VOF fraction F (Sec. 2 Eq. density with
 *     H(phi) = phi), optionally smoothed (1/4, 1/2, 1/4) along each axis (Sec. 2.10).
 * The solve is preconditioned conjugate gradients (Sec. 1); the paper names no preconditioner.
 *
 * Conventions shared by every entry point
 *   Layout   cells are numbered c = i + nx*(j + ny*k), x fastest.  Face arrays use the same order
 *            with the face axis one longer: x-faces (nz, ny, nx+1), y-faces (nz, ny+1, nx),
 *            z-faces (nz+1, ny, nx); x-face i lies between cells i-1 and i.
 *   Memory   unless stated otherwise every array argument is DEVICE memory, FP64, contiguous,
 *            owned by the caller, and only read during the call (outputs are written).  The
 *            library owns its workspace (coefficients, Krylov vectors, graphs) and frees it in
 *            vofp_destroy.
 *   Streams  all work is enqueued on the stream given to vofp_create.  Entry points that return
 *            a scalar (solve info, residual) synchronise that stream before returning.
 *   Errors   every call returns a vofp_status; VOFP_OK is 0.  No exception crosses the ABI, nothing
 *            calls exit or traps on the device.  vofp_last_error gives a message for the context.
 *            A failed solve still writes its best iterate and fills vofp_solve_info.
 *   Boundary domain faces are ordered -x, +x, -y, +y, -z, +z.  NEUMANN is a free-slip wall (no
 *            pressure flux unless neumann_flux prescribes one, Sec. 2.6 Eq. exit); DIRICHLET puts
 *            p = 0 on the face, half a cell from the adjacent centre.
 *   Cells    a cell has no unknown when its open volume is 0 or none of its flux-carrying faces
 *            is open; its faces are then closed and it reads 0 in every output.
 */
#ifndef VOFP_H
#define VOFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vofp_ctx vofp_ctx;
typedef struct vofp_nn vofp_nn;
/* A cudaStream_t (0 = legacy default stream). */
typedef struct CUstream_st* vofp_stream;

typedef enum {
    VOFP_OK = 0,
    VOFP_ERR_INVALID_ARG = 1,     /* bad pointer, size or option                                  */
    VOFP_ERR_CUDA = 2,            /* a CUDA runtime call failed (message in vofp_last_error)      */
    VOFP_ERR_OOM = 3,             /* device allocation failed                                     */
    VOFP_ERR_NOT_CONVERGED = 4,   /* max_iter reached before rtol (or 200 refinement steps)       */
    VOFP_ERR_BREAKDOWN = 5,       /* p.Ap <= 0, r.z <= 0 or a non-finite scalar in the iteration  */
    VOFP_ERR_STAGNATED = 6,       /* the iteration met rtol on its own residual but the residual  */
                                  /* recomputed from x stayed above rtol through restarts from x  */
    VOFP_ERR_INCOMPATIBLE_RHS = 7,/* all-Neumann problem whose right-hand side does not sum to 0  */
    VOFP_ERR_NOT_BUILT = 8,       /* vofp_build_operator has not succeeded on this context        */
    VOFP_ERR_DEVICE_TIMEOUT = 9   /* a bounded device-side wait (a bulk copy into shared memory)  */
                                  /* ran out after about one second; the solve stopped            */
} vofp_status;

enum { VOFP_BC_NEUMANN = 0, VOFP_BC_DIRICHLET = 1 };
enum { VOFP_MODE_FP64 = 0, VOFP_MODE_MIXED = 1, VOFP_MODE_FCG_NN = 2 };
enum { VOFP_PRECOND_JACOBI = 0, VOFP_PRECOND_RBSGS = 1 };

/* Grid: nx*ny*nz cells; dx, dy, dz are HOST arrays of the cell widths (lengths nx, ny, nz),
 * copied by vofp_create.  Stretched grids follow Sec. 2.2. */
typedef struct {
    int nx, ny, nz;
    const double* dx;
    const double* dy;
    const double* dz;
} vofp_grid;

/* Boundary kinds per domain face, and optional prescribed outward pressure flux
 * g = (1/rho) dp/dn on NEUMANN faces (device, one value per boundary face in the face's own
 * (row, column) order: -x/+x faces (nz, ny), -y/+y (nz, nx), -z/+z (ny, nx); NULL = 0).
 * The Orlanski exit of Sec. 2.6 (Eq. exit) is such a flux. */
typedef struct {
    int kind[6];
    const double* neumann_flux[6];
} vofp_bc;

/* Physical settings.  merge_threshold: cells with open-volume fraction below it merge into the
 * neighbour across their largest open face (Sec. 2.3 uses 0.25; 0 disables merging).
 * density_smoothing: 1 applies the filter of Sec. 2.10.  dt > 0 scales the right-hand side. */
typedef struct {
    double rho_liquid, rho_gas;
    double merge_threshold;
    int density_smoothing;
    double dt;
} vofp_phys;

/* Solve options.
 *   mode        VOFP_MODE_FP64: PCG in FP64.  VOFP_MODE_MIXED: iterative refinement whose outer
 *               residual b - A x and solution update are FP64 while the inner PCG runs with FP32
 *               coefficients and vectors and FP64-accumulated dot products.
 *   precond     VOFP_PRECOND_JACOBI (diagonal) or VOFP_PRECOND_RBSGS (red-black symmetric
 *               Gauss-Seidel, applied as CG on the black unknowns after eliminating the red ones
 *               (Eisenstat's form); both modes, and the bench default in mixed mode).
 *   rtol        the solve returns VOFP_OK only when the residual recomputed from the returned x,
 *               ||b_hat - A_hat x|| (2-norm over the unknowns, FP64), is at most rtol ||b_hat||.
 *               The iteration aims slightly below rtol; when the recomputed residual is still
 *               above rtol it restarts from x (a fresh residual), up to three times, each
 *               restart having to halve it (else VOFP_ERR_STAGNATED).
 *   max_iter    cap on PCG iterations (inner iterations summed in mixed mode).
 *   inner_rtol  mixed mode: relative residual reduction of each inner solve; 0 selects the
 *               default, 0.2 with inner_restart = 0 and 1e-3 with inner_restart = 1.
 *   inner_restart  mixed mode: 0 (default) keeps the FP32 search direction across refinement
 *               steps (the FP64 residual replaces the FP32 one, a "reliable update"); 1 restarts
 *               the inner PCG from p = r at every refinement step.
 *   check_every convergence is tested every check_every iterations (even, 2 .. 64; 0 = default:
 *               64 in mixed mode from 2^20 cells on, where an inner solve runs on to the end of
 *               its 64 iterations past its stop and saves refinement steps, 8 otherwise).
 *   x0_zero     1: ignore the contents of x and start from 0.
 *   host_loop   0: the loop runs as a CUDA graph with a device-side WHILE condition (no host round
 *               trip per iteration).  1: the host launches each kernel and reads the convergence
 *               flag every check_every iterations (same kernels and results; visible to profilers
 *               that do not trace conditional graph bodies).
 *   nn          VOFP_MODE_FCG_NN: a network bound to this operator (vofp_nn_bind).  The solve is
 *               FP64 iterative refinement whose inner solve is a flexible CG (FP32 vectors, FP64-
 *               accurate dots) preconditioned by the network, which also gives the initial guess.
 *               The network's steps continue while the inner residual norm falls at least to
 *               stag_ratio of its value stag_window iterations before; otherwise (or on a
 *               breakdown) the solve hands over to VOFP_MODE_MIXED (precond as given) from the
 *               current iterate.  A network application costs about as much as 30-40 iterations
 *               of the mixed red-black solve, so the defaults (window 2, ratio 0.6) keep it only
 *               while it beats those.
 *   stag_window, stag_ratio  the hand-over test above (0 selects the defaults; window <= 63). */
typedef struct {
    int mode;
    int precond;
    double rtol;
    int max_iter;
    double inner_rtol;
    int check_every;
    int x0_zero;
    int host_loop;
    vofp_nn* nn;
    int stag_window;
    int inner_restart;
    double stag_ratio;
} vofp_solve_opts;

typedef struct {
    int iterations;          /* PCG iterations (inner iterations summed in mixed mode)          */
    int outer_iterations;    /* refinement steps in mixed mode, 1 otherwise                     */
    double rel_residual;     /* ||b_hat - A_hat x|| / ||b_hat||, recomputed in FP64 at the end  */
    double seconds;          /* device time of the solve (CUDA events)                          */
    int status;              /* vofp_status of the solve                                        */
    int nn_applications;     /* network evaluations (VOFP_MODE_FCG_NN)                          */
    int fell_back;           /* 1 if VOFP_MODE_FCG_NN fell back to VOFP_MODE_MIXED              */
} vofp_solve_info;

typedef struct {
    long long cells;          /* nx*ny*nz                                                      */
    long long unknowns;       /* merge groups with an unknown                                  */
    long long inactive;       /* cells without an unknown                                      */
    long long merged_cells;   /* cells folded into another cell's unknown                      */
    long long groups;         /* merge groups with more than one cell                          */
    long long device_bytes;   /* device memory held by the context                             */
    int tma_stencil_fp32;     /* 1 if the FP32 CG stencil is fed by bulk tensor copies (TMA),  */
    int tma_stencil_fp64;     /* 0 for the register-prefetch kernel; both are set once the     */
                              /* context's kernels are prepared (first solve or timing call)   */
    int rb_compact;           /* 1 if the mixed red-black solve of this operator runs on       */
                              /* colour-compact vectors (set by its first solve or timing)     */
    int pdl_chained;          /* 1 if the kernels of the compact mixed iteration are chained   */
                              /* by programmatic dependent launch in the solve's graph (the    */
                              /* default; environment VOFP_PDL=0 turns it off, and the context */
                              /* turns it off if the driver refuses it inside the loop body)   */
} vofp_stats;

/* Library version string (static storage). */
const char* vofp_version(void);

/* Create a context for one grid on one stream.  *out receives the context.  Fails with
 * INVALID_ARG for non-positive sizes or widths, OOM if the grid arrays cannot be allocated. */
vofp_status vofp_create(vofp_ctx** out, const vofp_grid* grid, vofp_stream stream);

/* Free everything the context holds.  NULL is accepted. */
void vofp_destroy(vofp_ctx* ctx);

/* Message of the last failing call on ctx ("" if none; static text if ctx is NULL). */
const char* vofp_last_error(const vofp_ctx* ctx);

/* Assemble A_hat from the VOF fraction F (cells), the apertures ax, ay, az (faces, in [0,1]),
 * the open-volume fraction vol_frac (cells, in [0,1]; NULL = all 1), boundary kinds and physics
 * (Sec. 2 Eq. density; Sec. 2.3 Eqs. integral2 and merging; Sec. 2.10).  Computes cell activity,
 * the merge map (host side, O(number of small cells)), face coefficients and the scaled FP64 and
 * FP32 copies used by the solvers.  Synchronises the stream. */
vofp_status vofp_build_operator(vofp_ctx* ctx, const double* F, const double* ax,
                                const double* ay, const double* az, const double* vol_frac,
                                const vofp_bc* bc, const vofp_phys* phys);

/* b (cells) = -(1/dt) (sum of outward open-face fluxes A_f S_f u_f + body_flux) + prescribed
 * Neumann fluxes, for face velocities u (x-faces), v (y-faces), w (z-faces) (Sec. 2.1 Eq.
 * poisson1 with R = 0; Sec. 2.3 Eq. integral2).  body_flux (cells) is the integral of v*.n over
 * each cell's body surface (NULL = 0).  Normal velocities on NEUMANN domain faces are not used.
 * b is per cell and not merged; solve and residual merge it. */
vofp_status vofp_rhs_from_face_velocity(vofp_ctx* ctx, const double* u, const double* v,
                                        const double* w, const double* body_flux, double* b);

/* Projection of the face velocities (Sec. 2.1, Eq. runge1: u = u* - dt (1/rho) grad p) with the
 * operator's face reading (Sec. 2.3): on an interior face whose effective aperture is open,
 * u_out = u - dt (p_R - p_L) / ((d_L rho_L + d_R rho_R) / 2); on an open p = 0 domain face the
 * outside pressure 0 sits half a cell from the centre; on a free-slip domain face u_out = 0, or
 * -dt g on a + face and +dt g on a - face where an outward flux g = (1/rho) dp/dn was prescribed;
 * a closed face keeps u.  dt and rho are those of vofp_build_operator.
 *   p             device, cells: the pressure as vofp_solve returns it (every cell of a merge
 *                 group holds the group's value, 0 where there is no unknown).
 *   u, v, w       device, the x-, y- and z-face velocities u* (same layout as for the rhs).
 *   body_flux     device, cells, or NULL: as for vofp_rhs_from_face_velocity; enters div only.
 *   u_out, v_out, w_out  device, face arrays; may be u, v, w themselves (each face is read and
 *                 written by one thread).
 *   div           device, cells, or NULL: net outward flux of the projected field through each
 *                 cell's open faces plus body_flux, summed over each merge group at its master
 *                 (0 at the group's other cells and where there is no unknown).  With the exact
 *                 solution this vanishes: it is the residual of the pressure equation times -dt.
 *   max_div       host, or NULL: max |div| over cells (synchronises the stream).
 * Errors: NOT_BUILT before vofp_build_operator, INVALID_ARG for a null required pointer. */
vofp_status vofp_project(vofp_ctx* ctx, const double* p, const double* u, const double* v, const double* w,
                         const double* body_flux, double* u_out, double* v_out, double* w_out, double* div,
                         double* max_div);

/* Exit flux of the radiation condition (Sec. 2.6): from the x-momentum balance with the
 * Orlanski-type condition du/dt + u_c du/dx = 0 (Eq. orlanski), the pressure datum on the +x
 * domain face is (1/rho) dp/dx = u_c du/dx + R (Eq. exit).  Per exit face (row j, k; index
 * j + ny k) the call forms
 *     g = u_c (u[nx] - u[nx-1]) / dx[nx-1] + R - u[nx] / dt
 * from the x-face velocities u of that row (du/dx one-sided across the last cell; dt of
 * vofp_build_operator) and installs it as the prescribed flux of the +x face, which must be
 * NEUMANN in the built operator (copied into the context; later vofp_rhs_from_face_velocity and
 * vofp_project use it).  Free-slip faces take no normal velocity in the divergence and project to
 * -dt g on a + face, so the -u[nx]/dt term makes the projected exit velocity
 * u[nx] - dt (u_c du/dx + R): the discrete Orlanski update.
 *   u, v, w     device, face velocities (layout of vofp_rhs_from_face_velocity); v and w are read
 *               only when balance is set.
 *   body_flux   device, cells, or NULL (balance only).
 *   u_c         the ship's forward speed.
 *   R           device, (nz, ny) exit faces, or NULL (= 0): the remaining x-momentum terms R_1.
 *   balance     0: g as above.  1: g is then shifted by the same amount on every open exit face so
 *               that the right-hand side of the all-Neumann problem sums to zero (the radiation
 *               condition alone does not conserve mass); *shift receives the amount subtracted.
 *   g           device, (nz, ny), or NULL: a copy of the installed flux.
 *   shift       host, or NULL.
 * Errors: VOFP_ERR_NOT_BUILT before vofp_build_operator; VOFP_ERR_INVALID_ARG for a null u (or v,
 * w with balance) or a +x face that is not NEUMANN. */
vofp_status vofp_exit_flux(vofp_ctx* ctx, const double* u, const double* v, const double* w,
                           const double* body_flux, double u_c, const double* R, int balance, double* g,
                           double* shift);

/* VOF operator of Sec. 2.4, part 1: flux-error correction.  Face fluxes F = A (u - v) with A the
 * open face area (aperture x face area) and u, v, w the relative face velocities (u - v of the
 * paper); each cell's conservation error E = sum_i (F+_i - F-_i) (Eq. diverge) is removed along
 * z in proportion to the open areas of its two z faces (unchanged where both are closed); the
 * stage velocities u^_i = dx_i F~_i / V on the uncut faces are written to
 *   ux_hat   x faces (layout of u), uy_hat   y faces (layout of v),
 *   wm_hat, wp_hat   cells: the cell's own -z and +z face values (a z face shared by two cells may
 *                    carry two values after the correction).
 * ax, ay, az, u, v, w, outputs: device FP64.  Needs a context (grid), not a built operator. */
vofp_status vofp_vof_flux_correct(vofp_ctx* ctx, const double* ax, const double* ay, const double* az,
                                  const double* u, const double* v, const double* w, double* ux_hat,
                                  double* uy_hat, double* wm_hat, double* wp_hat);

/* VOF operator of Sec. 2.4: phi_out = phi - VOF(u, phi, dt).  The flux-error correction above,
 * then three operator-split stages along the axes (x, y, z) for order 0 or (z, y, x) for order 1
 * (the paper alternates them between time steps).  A stage moves fluid through the uncut faces
 * in slabs of thickness |u^| dt of the donor cell, cut by that cell's piecewise-linear interface
 * (normal = minus the gradient of phi by central differences weighted (1, 2, 1) x (1, 2, 1) over
 * the other two axes, skipping neighbours with vol_frac = 0 and outside the domain; plane position
 * from phi), and adds the dilation term dt phi (u^+ - u^-) / dx with the stage's new phi in the
 * first two stages and the stage's input phi in the third.  Inflow through a domain face takes the
 * boundary cell as donor; phi is not clipped; the caller keeps |u^| dt within a cell (the Courant
 * limit of Sec. 2.8).
 *   F            device, cells: phi at the start of the step.
 *   ax..w        device: apertures and relative face velocities (layouts of vofp_build_operator
 *                and vofp_rhs_from_face_velocity); vol_frac device, cells.
 *   dt > 0, order 0 or 1.
 *   F_out        device, cells; may be F itself.
 * Scratch (allocated on the first call, kept by the context): about 9 doubles per cell.
 * Needs a context (grid), not a built operator. */
vofp_status vofp_vof_advect(vofp_ctx* ctx, const double* F, const double* ax, const double* ay,
                            const double* az, const double* vol_frac, const double* u, const double* v,
                            const double* w, double dt, int order, double* F_out);

/* One second-order Runge-Kutta step of Sec. 2.1 around the pressure solve, from the library's own
 * calls on the context stream:
 *   stage 1: operator with rho(phi^k); P* from the face field u^k + dt R (Eq. poisson1), the solve
 *            starting from p; u* = u^k + dt (R - grad P* / rho) (Eq. runge1);
 *            phi* = phi^k - VOF(u^k, phi^k, dt);
 *   stage 2: operator with rho(phi*); P^{k+1} from the face field u* + u^k + dt R (Eq. poisson2),
 *            the solve starting from P*; u^{k+1} = (u* + u^k + dt (R - grad P^{k+1} / rho)) / 2
 *            (Eq. runge2); phi^{k+1} = phi^k - VOF((u* + u^k) / 2, phi^k, dt).
 * The right-hand side of each solve is -(1/dt) times the divergence of its face field and the
 * projection subtracts dt grad P / rho on the operator's faces (vofp_rhs_from_face_velocity,
 * vofp_project); VOF is vofp_vof_advect with the given axis order.
 *   F            device, cells: phi^k in, phi^{k+1} out.
 *   ax..vol_frac device: apertures and open volumes (as for vofp_build_operator).
 *   u, v, w      device, face velocities: u^k in, u^{k+1} out.
 *   Ru, Rv, Rw   device, face arrays of the momentum terms R, or all NULL (R = 0).
 *   bc, phys     as for vofp_build_operator (phys->dt is the step).
 *   opts         as for vofp_solve (x0_zero is ignored: both solves start from a pressure).
 *   p            device, cells: the first solve's starting guess in (the previous step's P^{k+1},
 *                or zeros), P^{k+1} out.
 *   order        0 or 1, the VOF axis order (alternate between steps).
 *   info         host, or NULL: both solves' vofp_solve_info and the largest group divergence of
 *                u^{k+1}.
 * Scratch: about 6 face arrays and 3 cell arrays, allocated on the first call.  Errors: those of
 * the calls it is made of; the step stops at the first failure (its arrays are then partly
 * updated). */
typedef struct {
    vofp_solve_info solve1, solve2;
    double max_div;
} vofp_rk2_info;
vofp_status vofp_rk2_step(vofp_ctx* ctx, double* F, const double* ax, const double* ay, const double* az,
                          const double* vol_frac, double* u, double* v, double* w, const double* Ru,
                          const double* Rv, const double* Rw, const vofp_bc* bc, const vofp_phys* phys,
                          const vofp_solve_opts* opts, double* p, int order, vofp_rk2_info* info);

/* y = A_hat x: x is read at each group's master cell; y receives the group's value at the master
 * and 0 at every other cell and at cells without an unknown. */
vofp_status vofp_apply(vofp_ctx* ctx, const double* x, double* y);

/* Merge b over groups and return ||b_hat - A_hat x|| / ||b_hat|| in *rel (FP64).  Synchronises. */
vofp_status vofp_residual(vofp_ctx* ctx, const double* b, const double* x, double* rel);

/* Solve A_hat x = b_hat (b per cell, merged internally).  x: initial guess on entry (unless
 * opts->x0_zero), solution on exit, with every cell of a group holding the group's value and 0
 * where there is no unknown.  info may be NULL.  Returns info->status. */
vofp_status vofp_solve(vofp_ctx* ctx, const double* b, double* x, const vofp_solve_opts* opts,
                       vofp_solve_info* info);

/* End-to-end call on HOST buffers (pageable or pinned): copies F, apertures, vol_frac and the
 * face velocities to the device, builds the operator, forms the right-hand side, solves and
 * copies the pressure back to x_host (cells).  Equivalent to the device-pointer calls above. */
vofp_status vofp_solve_host(vofp_ctx* ctx, const double* F, const double* ax, const double* ay,
                            const double* az, const double* vol_frac, const double* u,
                            const double* v, const double* w, const vofp_bc* bc,
                            const vofp_phys* phys, const vofp_solve_opts* opts, double* x_host,
                            vofp_solve_info* info);

/* One step of vofp_solve_host_batch: the inputs of vofp_solve_host (host buffers; vol_frac may be
 * NULL) and where that step's pressure goes. */
typedef struct vofp_host_step {
    const double* F;
    const double* ax;
    const double* ay;
    const double* az;
    const double* vol_frac;
    const double* u;
    const double* v;
    const double* w;
    double* x_host;
} vofp_host_step;

/* nsteps independent end-to-end solves on this context's grid, with one boundary set, physics and
 * options for all: step i gives the same x_host and infos[i] as vofp_solve_host on its buffers
 * (steps run in order; each builds the operator from its own inputs).  Step i + 1's uploads run
 * on a copy stream, into a second staging set, while step i solves (issued once its operator is
 * built), so with pinned host buffers a step costs about its device time plus the download of its
 * pressure; the copy stream waits for step 0's own uploads first.  Device staging: b and x (2 N
 * doubles) and two input sets of 2 N + 2 x (faces) doubles each, allocated on first use and kept
 * (one set with nsteps = 1).  infos: nsteps records, or NULL.  Returns OK, or the first
 * NOT_CONVERGED / BREAKDOWN among the steps (the batch goes on past those); any other error ends
 * the batch at that step, leaving its later x_host and infos untouched.  Every return comes after
 * the last copy that reads a caller's buffer.  vofp_solve_host is this call with one step. */
vofp_status vofp_solve_host_batch(vofp_ctx* ctx, int nsteps, const vofp_host_step* steps, const vofp_bc* bc,
                                  const vofp_phys* phys, const vofp_solve_opts* opts, vofp_solve_info* infos);

/* master[c] (device int32, cells) = root cell of c's merge group, -1 for cells without unknown. */
vofp_status vofp_merge_map(vofp_ctx* ctx, int32_t* master);

/* Counts and device memory of the built operator. */
vofp_status vofp_get_stats(vofp_ctx* ctx, vofp_stats* stats);

/* Same result as vofp_residual, for callers that must not allocate device memory after set-up:
 * code whose device memory belongs to another allocator (a framework's caching pool), a fixed
 * memory budget, or a loop that cannot take the device-wide synchronisation of cudaMalloc and
 * cudaFree.  vofp_residual may allocate the solver workspace on its first use; this call never
 * calls cudaMalloc, cudaFree or any allocating routine.  The paper has no counterpart: it is a
 * property of this library's interface.
 * Scratch: one file-scope device array of about 1 MB (every GPU that loads the library keeps it
 * until the process exits), enough for operators with at most 65536 merge groups; an operator with
 * more groups is rejected with VOFP_ERR_INVALID_ARG and a message.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  That first call is also where the CUDA runtime loads
 * this entry point's kernels and its array onto the device (lazy module loading, the default
 * since CUDA 12.2), a one-time reservation of about 1 MB plus code made by the runtime, not by
 * this call: make it during set-up, before a caching allocator takes the free device memory.
 * Later calls reserve nothing.  All calls share the array: calls that overlap on the GPU (other
 * streams or threads) race.  Synchronises the context stream; *rel is a host double. */
vofp_status vofp_residual_noalloc(vofp_ctx* ctx, const double* b, const double* x, double* rel);

/* Training pair in the scaled variables the solvers and the network use: r_scaled = S b_hat
 * (b merged over groups, S = diag(A_hat)^-1/2) and x_scaled = S^-1 x, both FP32 on every cell (0
 * without unknown; every cell of a group holds its group's value).  Device arrays. */
vofp_status vofp_scaled_pair(vofp_ctx* ctx, const double* b, const double* x, float* r_scaled, float* x_scaled);

/* ---- learned preconditioner (the paper has none; see VOFP_MODE_FCG_NN) --------------------
 * A 3-level 3-D convolutional encoder-decoder: two 3x3x3 convolutions with ReLU per level
 * (16, 32, 64 channels), 2x2x2 average pooling down, nearest upsampling up with skip
 * concatenation, and a 1x1x1 output layer.  Inputs per cell: the VOF fraction F, the mean open
 * fraction of the cell's x, y and z faces, log(dx/dx_min), log(dy/dy_min), log(dz/dz_min), and the
 * scaled residual divided by its RMS; the output is multiplied back by that RMS.  BF16
 * activations and weights on the tensor cores with FP32 accumulation; FP32 master weights trained
 * with Adam by the library's own forward and backward kernels.  Grid sizes must be multiples of 4.
 * Parameter order (get/set): per convolution layer its weights [27][cout][cin] then biases, for
 * the layers in forward order, then the output layer's 16 weights and its bias. */
vofp_status vofp_nn_create(vofp_nn** out, unsigned long long seed, vofp_stream stream);
void vofp_nn_destroy(vofp_nn* nn);
const char* vofp_nn_last_error(const vofp_nn* nn);
vofp_status vofp_nn_param_count(const vofp_nn* nn, long long* count);
/* host <- FP32 masters (grads = 0) or the gradients of the last vofp_nn_train_step (grads = 1) */
vofp_status vofp_nn_get_params(vofp_nn* nn, float* host, long long count, int grads);
vofp_status vofp_nn_set_params(vofp_nn* nn, const float* host, long long count);
/* geometry channels and the unknown mask from a built operator and its VOF fraction F (device) */
vofp_status vofp_nn_bind(vofp_nn* nn, vofp_ctx* ctx, const double* F);
/* copy the bound geometry out (geo: 8 BF16 per cell, device) / bind a stored one */
vofp_status vofp_nn_export_geometry(vofp_nn* nn, uint16_t* geo, float* mask);
vofp_status vofp_nn_set_geometry(vofp_nn* nn, int nx, int ny, int nz, const uint16_t* geo, const float* mask);
/* z = network(r) for a scaled residual r (device FP32, cells) */
vofp_status vofp_nn_forward(vofp_nn* nn, const float* r, float* z);
/* Check hooks for one 3x3x3 convolution layer (0..9, forward order) of the network, on caller
 * tensors of nx x ny x nz voxels (any positive sizes) in the network's chunk-planar BF16 layout:
 * channel c of voxel v (x fastest) at ((c / 8) * V + v) * 8 + c % 8, device memory, 16-byte aligned.
 * vofp_nn_conv_apply: data_grad = 0: out = ReLU(conv(in) + bias) with the layer's weights (in: its
 * input channels, out: its output channels); data_grad = 1: out = the data gradient of the
 * convolution applied to in (in: output channels, out: input channels; taps mirrored, no bias, no
 * ReLU).  vofp_nn_conv_wgrad: gw = dW[27][cout][cin] (tap index 9 (dz+1) + 3 (dy+1) + (dx+1)) =
 * sum over voxels of dy[v][co] x[v + tap][ci] and gb[cout] = sum over voxels of dy (FP32 device,
 * overwritten) from the layer input x and the output gradient dy.  These are the kernels the
 * forward pass and vofp_nn_train_step run; the paper has no counterpart.  VOFP_ERR_INVALID_ARG for
 * a bad layer, size, null or unaligned pointer; VOFP_ERR_DEVICE_TIMEOUT if a bounded wait ran
 * out. */
vofp_status vofp_nn_conv_apply(vofp_nn* nn, int layer, int data_grad, int nx, int ny, int nz, const uint16_t* in,
                               uint16_t* out);
vofp_status vofp_nn_conv_wgrad(vofp_nn* nn, int layer, int nx, int ny, int nz, const uint16_t* x, const uint16_t* dy,
                               float* gw, float* gb);
/* forward, masked mean-squared error against target (both relative to the RMS of r), backward;
 * update = 1 also takes an Adam step with learning rate lr.  *loss (host) may be NULL. */
vofp_status vofp_nn_train_step(vofp_nn* nn, const float* r, const float* target, float lr, int update,
                               float* loss);

/* Training step of the network as a preconditioner of ctx's operator (the network bound to ctx's
 * grid): r is a scaled residual and e the exact error it leaves (FP32 device cells, scaled
 * variables as in vofp_scaled_pair, A_scaled e = r).  The loss is the relative A-norm error of the
 * network output z, (z - e)' A_scaled (z - e) / (e' A_scaled e) over the unknowns (1 for z = 0),
 * whose gradient 2 (A_scaled z - r) / (e' r) needs one operator apply; then backward and, with
 * update = 1, an Adam step with learning rate lr.  *loss (host) may be NULL.  Runs on ctx's stream
 * and synchronises it.  The paper has no counterpart. */
vofp_status vofp_nn_train_step_anorm(vofp_nn* nn, vofp_ctx* ctx, const float* r, const float* e, float lr,
                                     int update, float* loss);

/* *count = number of kernels this context has launched since vofp_create (kernels run inside
 * the solve's CUDA graphs are counted per execution). */
vofp_status vofp_launch_count(vofp_ctx* ctx, long long* count);

/* Measurement hook: after a vofp_solve, launches one CG iteration's kernels `reps` times each on
 * the context stream -- FP64 (precision 64) or FP32 (precision 32), Jacobi or red-black (precond)
 * -- and records the average device time of the fused stencil kernel in *stencil_ms, of the
 * vector-update kernel in *update_ms and, for the FP32 red-black iteration on colour-compact
 * vectors (else 0), of its fix-row and merge-group kernel in *aux_ms (the exception rows run
 * inside the stencil kernel there).  Step
 * sizes are held at zero, so every byte is read and written but the vectors keep their values;
 * the solution returned by the solve is untouched. */
vofp_status vofp_time_iteration_kernels(vofp_ctx* ctx, int precision, int precond, int reps,
                                        float* stencil_ms, float* update_ms, float* aux_ms);

/* Measurement hook (no context): the current device's fused multiply-add throughput in FP64 and
 * FP32, in TFLOP/s (two flops per FMA), from a kernel of independent FMA chains on every SM timed
 * with CUDA events on `stream` (best of three launches after a warm-up; about 40 ms in all).  It
 * is the roof of kernels bound by the FP64 pipe (the FP64 CG iteration, the VOF stages); the paper
 * has no counterpart.  Synchronises the stream.  VOFP_ERR_INVALID_ARG for null outputs,
 * VOFP_ERR_CUDA if a launch or event call fails. */
vofp_status vofp_measure_fma_peaks(vofp_stream stream, double* fp64_tflops, double* fp32_tflops);

/* Host-only planning query (no context, no device): how the colour-compact red-black iteration
 * kernel splits its work over `slots` resident blocks for tiles_x x tiles_y tiles (32 pairs x 16
 * rows each by default) and nz planes.  The tiles form groups of *gx x *gy neighbours (*gx divides
 * tiles_x, *gy divides tiles_y); block b is member b % (gx gy) of group g = b / (gx gy), which
 * marches the work items [g per, (g+1) per) of w = column (nz + pad) + pad + plane over the
 * (tiles_x / gx) x (tiles_y / gy) group columns (x-fastest; the first `pad` items of a column
 * stand for no plane); member m takes tile (column x gx + m % gx, column y gy + m / gx).
 * *blocks = number of blocks (<= slots, a multiple of gx gy).  The plan minimises the plane steps
 * of the costliest block (each column segment adds five steps to its planes) weighted by the DRAM
 * bytes of the tile edges whose two sides are not marched at the same plane in the same step
 * (inside a group they always are; their halo otherwise comes from DRAM instead of L2).
 * VOFP_ERR_INVALID_ARG for null outputs, non-positive sizes, or more work items than an int
 * holds.  (The library's own plan takes the group from VOFP_RBC_GROUP="gx,gy" when set.) */
vofp_status vofp_rbc_split_plan(int tiles_x, int tiles_y, int nz, int slots, int* blocks, int* per, int* pad,
                                int* gx, int* gy);

#ifdef __cplusplus
}
#endif
#endif /* VOFP_H */
