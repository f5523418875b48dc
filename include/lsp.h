/*
 * lsp.h -- C ABI of the GB300 (sm_103a) explicit Hamilton-Jacobi level-set
 * integrator.  The method is the one of "LevelSetPy" (arXiv 2411.03501):
 * explicit integration of  phi_t + H(x, grad phi) = 0  (Eq. 1) on a dense
 * Cartesian grid with ghost-cell boundaries (Sec. III-B), upwind ENO/WENO
 * one-sided derivatives (Sec. IV-A..IV-C), the Lax-Friedrichs numerical
 * Hamiltonian with global-LF dissipation (Sec. IV-D, Listing 4), a CFL time
 * step (Sec. IV-D, V-A), TVD-RK1/2/3 (Sec. V-A) and, for reachable tubes,
 * the minimum with the target after each step (Sec. VI-A, Eq. 30).
 *
 * Conventions shared by every call:
 *  - Fields are dense C-order arrays (last axis fastest) of n[0]*...*n[d-1]
 *    elements of the solve's dtype (float or double), in DEVICE memory of the
 *    current CUDA device, 16-byte aligned.  The caller owns every field and
 *    every workspace; the library owns only its opaque handles and never
 *    allocates device memory inside a step or a solve.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; calls return without waiting for the
 *    GPU unless stated otherwise.
 *  - Sign convention: phi_t + H = 0 integrated forward in time-to-go.
 *    Reachability Hamiltonians are H = -max_u min_d p.f (Eq. 31).
 *  - Every call returns an lsp_status and never aborts the process.  The
 *    text of the last error of the calling thread is in lsp_last_error().
 *    Asynchronous CUDA errors surface as LSP_ECUDA on a later call.
 *  - Device-side failures (non-finite values produced, a bounded wait that
 *    ran out) set a flag in the workspace; they are reported when the call
 *    waits for the GPU (lsp_solve_opts.check_finite) or by
 *    lsp_check_status().  No kernel of the library spins without a limit.
 */
#ifndef LSP_H
#define LSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSP_OK = 0,
    LSP_EINVAL = 1,       /* bad argument (described by lsp_last_error)      */
    LSP_ENOMEM = 2,       /* workspace too small                             */
    LSP_ECUDA = 3,        /* a CUDA runtime error                            */
    LSP_EUNSUPPORTED = 4, /* combination not provided                       */
    LSP_ENONFINITE = 5,   /* a NaN or infinity was produced                  */
    LSP_ETIMEOUT = 6      /* a bounded device-side wait gave up              */
} lsp_status;

/* Boundary condition of one axis (Sec. III-B: boundary conditions are set
 * by populating ghost cells).  PERIODIC wraps around (the axis' upper bound
 * is then the image of the lower one and is not a node).  EXTRAPOLATE fills
 * ghost cells by linear extrapolation from the two nodes nearest the
 * boundary. */
typedef enum { LSP_BC_EXTRAPOLATE = 0, LSP_BC_PERIODIC = 1 } lsp_bc;

/* One-sided derivative approximation (the CoStateCalc of Listing 4):
 * first-order upwinding (Sec. IV-A), ENO2 and ENO3 (Sec. IV-B), HJ-WENO5
 * (Sec. IV-C).  Ghost widths 1, 2, 3, 3. */
typedef enum { LSP_UPWIND1 = 0, LSP_ENO2 = 1, LSP_ENO3 = 2, LSP_WENO5 = 3 } lsp_scheme;

/* Dynamics (hamFunc + partialFunc of Listing 4).  Parameters:
 *  NORMAL_SPEED  any d   H = a |p|                            {a}
 *  TRANSLATE     any d   H = v . p                            {v_0..v_{d-1}}
 *  QUADRATIC     any d   H = |p|^2 / 2 (LF bound from p)      {}
 *  AIR3D         d = 3   relative pursuit-evasion (x, y, theta); evader
 *                        turn rate u maximises, pursuer turn rate d
 *                        minimises; H = -max_u min_d p.f      {v_e, v_p, u_max, d_max}
 *  CAR4D         d = 4   car (x, y, theta, v), turn rate and
 *                        acceleration minimise p.f (reach)     {w_max, a_max}
 *  ROCKETS       d = 3   two rockets (Sec. VI-A, Eq. 31), relative
 *                        (x, z, theta): f = (a cos th + u_e x,
 *                        a sin th + a + u_p x - g, u_p - u_e); evader
 *                        thrust angle u_e in [-ue, ue] maximises,
 *                        pursuer u_p in [-up, up] minimises    {a, g, ue, up}
 *  DOUBLE_INTEGRATOR d = 2  x1dot = x2, x2dot = u, |u| <= umax,
 *                        u minimises p.f (reach)                {umax}
 * The adjoint covers every dynamics but QUADRATIC (whose LF bound depends
 * on the costate).
 */
typedef enum {
    LSP_DYN_NORMAL_SPEED = 0,
    LSP_DYN_TRANSLATE = 1,
    LSP_DYN_QUADRATIC = 2,
    LSP_DYN_AIR3D = 3,
    LSP_DYN_CAR4D = 4,
    LSP_DYN_ROCKETS = 5,
    LSP_DYN_DOUBLE_INTEGRATOR = 6
} lsp_dyn;

typedef enum { LSP_F32 = 0, LSP_F64 = 1 } lsp_dtype;

/* Dissipation coefficients of the Lax-Friedrichs term (Sec. IV-D).  GLF:
 * alpha_k is the grid maximum of the bound on |dH/dp_k| (the routine the
 * paper's Listing 4 names).  LLF / LLLF: the bound at each node, over the
 * node's own costate interval in dimension k (LLF) or in every dimension
 * (LLLF) and the global interval elsewhere.  The bounds of the dynamics
 * provided involve at most the costate of their own dimension, so LLF and
 * LLLF coincide for them.  The CFL step uses the grid maxima, which are the
 * GLF coefficients in every mode. */
typedef enum { LSP_DISS_GLF = 0, LSP_DISS_LLF = 1, LSP_DISS_LLLF = 2 } lsp_diss;

typedef struct lsp_grid lsp_grid; /* opaque: grid + dynamics */

/* Options of a step or a solve (the odeCFLx options of Listing 3). */
typedef struct {
    int rk_order;      /* 1, 2 or 3 (TVD-RK, Sec. V-A)                     */
    int scheme;        /* lsp_scheme                                       */
    int dtype;         /* lsp_dtype of phi, target and the workspace fields */
    int tube;          /* 1: phi <- min(phi, target) after every step      */
    double cfl;        /* CFL number in (0, 1]                             */
    int check_finite;  /* 1: wait for the GPU at the end of the call and
                          return LSP_ENONFINITE if a non-finite value was
                          produced                                         */
    int use_graph;     /* 1: lsp_hj_solve replays its launches as a CUDA
                          graph (captured on the first call with the same
                          arguments, kept in the grid handle);
                          lsp_hj_solve_batched captures its launches into
                          one graph and launches that                      */
    int batch_chunk;   /* batched solves: planes per CTA along the march of
                          3-D/4-D problems (0 = 128)                        */
    int batch_persistent; /* batched solves: 1 = the whole solve as ONE
                          launch of resident CTAs that take (step, stage,
                          tile) items in order and wait on per-problem
                          completion counters (use_graph ignored)          */
    int batch_wait_ms; /* persistent batched solves: limit of one device
                          wait in milliseconds (0 = 1000); a wait that runs
                          out ends the launch with LSP_ETIMEOUT            */
    int diss;          /* lsp_diss (0 = GLF)                               */
    int varform;       /* 1: the variational form of the reachable-tube PDE
                          (Eq. 30: phi_t + min[0, H] = 0 in the paper's
                          backward time; here every stage rate L = -Hhat is
                          replaced by min(L, 0), so phi never increases).
                          Independent of tube.                             */
    int batch_tiles;   /* batched solves: tile of the two fastest axes of
                          the d-dimensional problems in bits 2(d-2)..2(d-2)+1:
                          0 = 16 x 16 nodes, 1 = 32 x 8, 2 = 64 x 4 (every
                          CTA has 256 threads); 0 = 16 x 16 for every
                          dimension; lsp_batched_autotune picks them; with
                          local coefficients or the clip the tiles are
                          16 x 16 whatever this says                       */
} lsp_solve_opts;

typedef struct {
    int64_t steps;     /* RK steps taken                                   */
    int64_t stages;    /* stage evaluations (steps * rk_order)             */
    double dt_min;     /* smallest and largest step                        */
    double dt_max;
    double t_end;      /* time reached (FP64 accumulator)                  */
} lsp_solve_stats;

/* Create a grid (createGrid(gmin, gmax, N, pdim) of Listing 1).
 *  ndim      1..4
 *  gmin/gmax ndim lower / upper bounds (host), finite, gmax > gmin
 *  n         ndim node counts (host), each >= 7 (room for a 3-cell stencil)
 *  bc        ndim boundary conditions (host), lsp_bc values
 * Spacing: (gmax-gmin)/(n-1) on non-periodic axes, (gmax-gmin)/n on periodic
 * ones.  *out receives a handle to be released with lsp_grid_destroy.
 * Errors: LSP_EINVAL on a bad argument; nothing is allocated then. */
lsp_status lsp_grid_create(int ndim, const double* gmin, const double* gmax, const int64_t* n,
                           const int* bc, lsp_grid** out);

/* Release a grid and anything cached in it (captured graphs).  NULL is a
 * no-op. */
void lsp_grid_destroy(lsp_grid* grid);

/* Attach dynamics to a grid (the hamFunc / partialFunc / dissFunc triple of
 * Listing 4).  params: nparams doubles (host), see lsp_dyn.  For dynamics
 * whose bound on |dH/dp_k| depends on the state only, the global-LF
 * coefficients alpha_k = max over the grid nodes of that bound are computed
 * here on the current device (a reduction kernel; the call waits for it).
 * Errors: LSP_EINVAL (wrong parameter count, dimension mismatch, non-finite
 * parameter), LSP_ECUDA. */
lsp_status lsp_set_dynamics(lsp_grid* grid, int dyn, const double* params, int nparams);

/* The global-LF coefficients alpha_k (host, ndim doubles) found by
 * lsp_set_dynamics.  LSP_EUNSUPPORTED for QUADRATIC (its alpha depends on
 * phi and is recomputed on the device at every stage). */
lsp_status lsp_get_alpha(const lsp_grid* grid, double* alpha);

/* Bytes of device workspace a step or solve with these options needs: two
 * stage fields (one for RK1/RK2) plus a 256-byte control block. */
lsp_status lsp_workspace_size(const lsp_grid* grid, const lsp_solve_opts* opts, size_t* bytes);

/* The CFL step of Sec. IV-D / V-A for time t:
 *   dt = min(cfl / sum_k(alpha_k / dx_k), t_final - t)   (FP64, host)
 * Not available for QUADRATIC (LSP_EUNSUPPORTED). */
lsp_status lsp_cfl_dt(const lsp_grid* grid, const lsp_solve_opts* opts, double t,
                      double t_final, double* dt);

/* Method-of-lines rate L(phi) = -Hhat at every node (Sec. IV-D and V-A):
 *   Hhat = H(x, (p^+ + p^-)/2) - sum_k alpha_k (p^+_k - p^-_k) / 2
 * with p^-/p^+ from opts->scheme and alpha the global-LF coefficients.
 * phi (in), rate (out): device fields of opts->dtype.  Uses the workspace
 * control block.  Asynchronous. */
lsp_status lsp_hj_rate(lsp_grid* grid, const lsp_solve_opts* opts, const void* phi, void* rate,
                       void* workspace, size_t workspace_bytes, void* stream);

/* One TVD-RK step (Sec. V-A) of phi in place, followed, if opts->tube, by
 * phi <- min(phi, target) (Sec. VI-A).  Each stage is one fused kernel:
 * ghost cells, derivatives, Hamiltonian + LF, RK combination (and the
 * minimum with the target in the last stage).
 *  phi       device field, in/out
 *  target    device field (read if opts->tube, else may be NULL)
 *  t         time of phi (only for the CFL step)
 *  dt_io     in: step size if *dt_io > 0; if *dt_io <= 0 the CFL step for
 *            t_final = +inf is used and written back (not for QUADRATIC,
 *            whose step the device computes; *dt_io then must be <= 0 and
 *            receives the step after waiting for the GPU).
 * Errors: LSP_EINVAL, LSP_ENOMEM (workspace too small), LSP_ECUDA,
 * LSP_ENONFINITE (only with opts->check_finite). */
lsp_status lsp_hj_step(lsp_grid* grid, const lsp_solve_opts* opts, void* phi,
                       const void* target, double t, double* dt_io, void* workspace,
                       size_t workspace_bytes, void* stream);

/* Integrate phi in place from t0 to t_final (odeCFLx of Listing 3): CFL
 * steps of dt = min(cfl / sum_k alpha_k/dx_k, t_final - t), the time kept
 * in FP64, stopping once t >= t_final - 1e-12 |t_final|.  Arguments as for
 * lsp_hj_step; stats (host, nullable) receives the step count and range.
 * For state-only bounds the step sequence is known on the host, so the
 * call only enqueues work (or replays a captured graph with
 * opts->use_graph).  For QUADRATIC it waits for the GPU once per step. */
lsp_status lsp_hj_solve(lsp_grid* grid, const lsp_solve_opts* opts, void* phi,
                        const void* target, double t0, double t_final, void* workspace,
                        size_t workspace_bytes, lsp_solve_stats* stats, void* stream);

/* Tile of the tiled stage kernel used for FP32 grids of 3 or 4 dimensions
 * (the generic one-thread-per-node kernel serves every other case).  A CTA
 * of tb x ta threads covers tb nodes of the fastest axis and ta of the
 * second fastest and marches along the third over ch planes; each plane of
 * the tile is staged in shared memory with a 3-cell halo.  minb (2, 3 or 4)
 * selects the kernel variant compiled for that many CTAs per SM (register
 * budget 128, 80 or 64 per thread); pair = 1 (WENO5, ENO2, ENO3) selects
 * the variant that carries two consecutive planes per thread through paired
 * FP32 instructions, pair = 2 (WENO5 only) the same with the marching axis'
 * WENO5 terms evaluated once per face (shared by the two nodes of the face;
 * results identical to pair = 1 bit for bit).  pair = 3 (ENO2 and ENO3)
 * selects the face-shared ENO kernel: each thread owns 4 consecutive nodes
 * of the fastest axis, so a CTA has tb/4 x ta threads and tb is 16, 28 or
 * 32; every ENO stencil choice is made once per cell face for both nodes of
 * the face (along the fastest axis within a thread's run, along the
 * marching axis in a register pipeline); minb is 2 (128 registers) for it.
 * pair = 4 is the same with runs of 2 nodes (tb/2 x ta threads, minb 3: 80
 * registers, more resident warps).
 * Its results agree with the other variants to FP32 rounding, not bit for
 * bit (the same selections, the arithmetic grouped differently).
 * pair = 5 (3-D grids, any scheme) is temporal blocking of TVD-RK2: both
 * stages of a step in one launch, the first stage evaluated in shared memory
 * on the tile plus its halo (G cells along the tile axes, G planes at each
 * end of the chunk) and the second on the tile, with the same operations
 * as the scalar body (pair 0), so the result equals two scalar-body stages.
 * It serves RK2 steps and solves with GLF dissipation, no clip and dynamics
 * with state-only bounds; lsp_hj_solve then alternates phi and the
 * workspace's stage field (copying the result to phi at the end when the
 * step count is odd), lsp_hj_step writes the stage field and copies it
 * back.  Every other stage on such a tile (RK1, RK3, lsp_hj_rate, the
 * adjoint's forward) runs the scalar body of the same tile.  lsp_autotune
 * does not try it.  A tile
 * whose pair the scheme
 * has no variant for makes the step use the generic kernel.  With local
 * dissipation coefficients or the variational clip (opts->diss, varform),
 * pair = 2 runs its local variant when the dynamics' bounds depend on the
 * state only (every dynamics but QUADRATIC); other tiles run the scalar
 * body with the local coefficients and the clip.
 *  lsp_set_tile(g, 0, 0, 0, 0, 0)   default: WENO5 16 x 16, 3 CTAs/SM, pair 2,
 *                                   chunks for ~3 waves (even length); other
 *                                   schemes 32 x 8, 3 CTAs/SM, chunks for ~2
 *                                   waves
 *  lsp_set_tile(g, -1, 0, 0, 0, 0)  always use the generic kernel
 *  lsp_set_tile(g, tb, ta, ch, minb, pair) explicit; LSP_EINVAL unless
 *        the launch has <= 65535 z-blocks, minb is 2, 3 or 4 and either
 *        pair is 0, 1 or 2 with tb*ta <= 256 and the haloed tile fitting 3
 *        values per thread, or pair is 3 (4) with tb in {16, 28, 32},
 *        (tb/4)*ta <= 256 ((tb/2)*ta <= 256) and two staged planes within
 *        200 KB of shared memory, or pair is 5 on a 3-D grid with tb*ta <=
 *        256, the tile with a 4-cell halo fitting 4 values per thread and
 *        with a 2-cell halo 3 (checked for ENO2; a step whose scheme's
 *        halo does not fit runs the generic kernel).
 * lsp_get_tile reports the tile a step with `opts` would use (all -1 when
 * the generic kernel runs). */
lsp_status lsp_set_tile(lsp_grid* grid, int tb, int ta, int ch, int minb, int pair);
lsp_status lsp_get_tile(const lsp_grid* grid, const lsp_solve_opts* opts, int* tb, int* ta,
                        int* ch, int* minb, int* pair);

/* Autotuner: time whole RK steps of the solve on a scratch copy of phi
 * (phi is not modified; a copy of phi stands in for the tube target; two
 * fields are allocated for the call, and without room for them the first
 * stage alone is timed) for a set of tile shapes (7 fixed, 2 fitted to the
 * grid), chunk lengths, occupancy targets and kernel variants (WENO5: pair 0,
 * 1, 2; ENO2 and ENO3: pair 0, 1, plus the face-shared runs of pairs 3 and
 * 4 on 3 widths x 6 row counts x 7 chunk lengths), re-time the
 * six fastest over longer windows and keep the best in the grid handle
 * (reported through tb/ta/ch/minb/pair, which may be NULL).  Waits for the
 * GPU.  For grids without a tiled kernel it selects the generic one (all
 * -1).  LSP_EUNSUPPORTED for QUADRATIC. */
lsp_status lsp_autotune(lsp_grid* grid, const lsp_solve_opts* opts, const void* phi,
                        void* workspace, size_t workspace_bytes, void* stream, int* tb, int* ta,
                        int* ch, int* minb, int* pair);

/* lsp_hj_solve without a workspace argument, for callers that cannot
 * allocate device memory: for example a real-time control loop that must
 * not call cudaMalloc/cudaFree (they can block and synchronise the whole
 * device), or a host whose device memory is entirely owned by another
 * allocator (a framework's caching allocator, a fixed arena) and so has no
 * buffer to hand over.  The paper has no counterpart: this is a property of
 * the library, not of the method.
 *  - Scratch lives in a static 32 MiB device array inside the library (held
 *    on every GPU that loads the library until the process exits); grids
 *    whose lsp_workspace_size exceeds 32 MiB are rejected with LSP_ENOMEM
 *    and a message giving both sizes (FP32 RK3: up to ~4.19M nodes).
 *  - The first call on a device looks up the array's device address (a
 *    one-time set-up with that device current) and keeps it for the life of
 *    the process; make that first call before any stream capture.  Because
 *    the address is kept per device index, resetting the device
 *    (cudaDeviceReset) or making a non-primary context current on it after
 *    that first call is not supported: the module is then loaded again at
 *    another address and the kept one is stale.
 *  - Every call in a process shares the one array, which keeps the last
 *    call's contents (the solve never reads them: flags are cleared on entry
 *    and stage fields are written before being read).  Calls in one process
 *    whose GPU work overlaps (different streams or host threads) race on it:
 *    serialise them.  Separate processes each have their own copy of the
 *    array (one per CUDA context) and do not interfere.
 *  - opts->use_graph must be 0.  Other arguments, results and errors as for
 *    lsp_hj_solve.  Nothing is allocated. */
lsp_status lsp_hj_solve_noalloc(lsp_grid* grid, const lsp_solve_opts* opts, void* phi,
                                const void* target, double t0, double t_final,
                                lsp_solve_stats* stats, void* stream);

/* Autotuner of the batched solve's tiles: times the batched solve of these
 * problems over a short horizon (at most 8 CFL steps each, on scratch
 * copies of phis: the caller's fields are not modified; the copies are
 * allocated for the call) for the tile shapes of opts->batch_tiles, one
 * problem dimension at a time (coordinate descent from opts->batch_tiles),
 * and returns the fastest in *batch_tiles for the caller to store in
 * opts->batch_tiles.  Arguments as for lsp_hj_solve_batched; the workspace
 * from lsp_batched_workspace_size serves every tile choice.  Waits for the
 * GPU. */
lsp_status lsp_batched_autotune(int nprob, lsp_grid* const* grids, const lsp_solve_opts* opts,
                                const void* const* phis, const void* const* targets,
                                const double* t_final, void* workspace, size_t workspace_bytes,
                                void* stream, int* batch_tiles);

/* Batched solves: nprob independent problems (own grid, dynamics, CFL step
 * and t_final each) advanced together, problem i from t = 0 to t_final[i].
 * One kernel launch advances one RK stage of every problem that still has
 * steps left; CTAs map to (problem, tile) through a table in the workspace,
 * so problems of different sizes and dimensions share every launch.
 *  grids    nprob grids with state-only LF bounds (NORMAL_SPEED, TRANSLATE
 *           in 2-4 D, AIR3D, CAR4D)
 *  opts     shared: FP32, RK2 or RK3, scheme, CFL, tube, use_graph,
 *           batch_chunk
 *  phis     nprob device fields (in/out), targets: nprob device fields
 *           (read if opts->tube)
 *  t_final  nprob final times (host)
 *  stats    nprob entries (host, nullable)
 * Workspace: lsp_batched_workspace_size bytes (control block, problem
 * table, CTA table, persistent-launch state, two stage fields per problem).
 * Each problem's result equals the single-problem solve of the same grid to
 * FP32 rounding.
 *
 * opts->batch_persistent = 1 runs the same stages as ONE cooperative launch
 * of as many CTAs as fit on the device at once.  The CTAs take work items
 * (step, stage, tile) from one counter in that order; an item waits until
 * every tile of the previous stage of its problem has been counted done, so
 * problems advance independently (a short problem is not held back by the
 * launch boundaries of a long one) and no host launch separates stages.
 * Every tile computes exactly what the stage-synchronous launch computes
 * (identical results bit for bit).  Each wait is bounded by
 * opts->batch_wait_ms; one that runs out raises LSP_ETIMEOUT (reported as
 * described for check_finite), makes the other CTAs stop at their next item
 * and leaves the fields partly advanced; the CUDA context stays usable. */
lsp_status lsp_batched_workspace_size(int nprob, lsp_grid* const* grids,
                                      const lsp_solve_opts* opts, size_t* bytes);
lsp_status lsp_hj_solve_batched(int nprob, lsp_grid* const* grids, const lsp_solve_opts* opts,
                                void* const* phis, const void* const* targets,
                                const double* t_final, void* workspace, size_t workspace_bytes,
                                lsp_solve_stats* stats, void* stream);

/* Discrete adjoint of a solve with a FIXED number of steps nsteps (dt from
 * the CFL condition of the state-only GLF coefficients, no shortened last
 * step), with sqrt(N) checkpointing.  The reverse replays every stage with
 * the forward's selections frozen -- ENO stencils, the argmax inside the
 * WENO regulariser, the signs of the optimal inputs, the min with the
 * target, the grid node attaining each GLF coefficient -- and differentiates
 * the rest exactly (the WENO weights included).  Dynamics parameters act
 * through H, through the GLF coefficients and through dt.
 *
 * lsp_adjoint_workspace_size: bytes for ncheck checkpoints (0: ceil(sqrt
 *   nsteps)), a segment of ceil(nsteps/ncheck) recomputed states with the
 *   RK stage inputs of each (rk_order - 1 fields per state, kept by the
 *   recomputation for the reverse sweep), the stage fields, five adjoint
 *   fields and 7*ndim coefficient fields.  ncheck < 0 keeps everything:
 *   the forward stores every state and every stage input (nsteps * rk_order
 *   fields) and the reverse sweep recomputes nothing -- the fastest form
 *   where memory allows (air3d 129^3, 200 RK3 steps: 5.2 GB in FP32).
 * lsp_hj_solve_ckpt: the forward solve (phi in place), storing checkpoints
 *   in the workspace.  Asynchronous.
 * lsp_hj_adjoint: the reverse sweep from the checkpoints left in the same
 *   workspace by lsp_hj_solve_ckpt (same grid, dynamics, opts, nsteps,
 *   ncheck, target).
 *   lamT        dLoss/dphi(t_end), device field (in)
 *   lam0        dLoss/dphi0, device field (out)
 *   lam_target  dLoss/dtarget, device field (out, nullable; tube only)
 *   dprm        dLoss/dparams, 8 host doubles (out; the lsp_set_dynamics
 *               parameters in order, the rest zero)
 *   Waits for the GPU (reads the parameter accumulators).
 * Not for QUADRATIC (LSP_EUNSUPPORTED). */
lsp_status lsp_adjoint_workspace_size(const lsp_grid* grid, const lsp_solve_opts* opts,
                                      int nsteps, int ncheck, size_t* bytes);
lsp_status lsp_hj_solve_ckpt(lsp_grid* grid, const lsp_solve_opts* opts, void* phi,
                             const void* target, int nsteps, int ncheck, void* workspace,
                             size_t workspace_bytes, void* stream);
lsp_status lsp_hj_adjoint(lsp_grid* grid, const lsp_solve_opts* opts, const void* target,
                          int nsteps, int ncheck, const void* lamT, void* lam0, void* lam_target,
                          double* dprm, void* workspace, size_t workspace_bytes, void* stream);

/* Loss of the differentiation workload and its gradient:
 *   value = sum_i H_eps(-phi_i) dV + sum_q phi(x_q),
 *   H_eps(s) = 1 / (1 + exp(-s/eps)), eps = max_k dx_k, dV = prod_k dx_k,
 * phi(x_q) by multilinear interpolation at nq query states (device, nq x ndim
 * row-major, same dtype; periodic axes wrap, others clamp).  value_dev: one
 * device double (overwritten); grad: device field (overwritten, nullable).
 * Asynchronous. */
lsp_status lsp_loss_tube(const lsp_grid* grid, int dtype, const void* phi, const void* queries,
                         int nq, double* value_dev, void* grad, void* stream);

/* Implicit surfaces (Sec. III-C, III-D): fields built on the device, for
 * targets and initial conditions.  Each primitive writes, at every node of
 * `grid` (coordinates lo + i dx, C order), a value whose zero level set is
 * the shape and which is negative inside; distances are measured in the
 * dimensions whose bit is clear in `ignore_mask` (bit k = dimension k), so
 * ignoring dimensions extrudes the shape along them (a sphere becomes a
 * cylinder).  Periodic axes are not wrapped.  Arithmetic in `dtype`; `out`
 * is a device field of the grid's size.  Asynchronous.
 *  lsp_shape_sphere     |x - center| - radius (signed distance)
 *  lsp_shape_box        signed distance to the box [lo, hi] (exact: the
 *                       Euclidean distance outside, minus the distance to
 *                       the nearest face inside)
 *  lsp_shape_quadric    sum_k w_k (x_k - center_k)^2 - offset: the
 *                       ellipsoid form of Sec. III-C (not a distance)
 *  lsp_shape_halfspace  n . (x - point) / |n| (signed distance to the plane;
 *                       polyhedra are intersections of half spaces)
 * LSP_EINVAL for a NULL pointer, an unset grid, all dimensions ignored, a
 * negative radius, lo > hi or a zero normal. */
lsp_status lsp_shape_sphere(const lsp_grid* grid, int dtype, const double* center, double radius,
                            unsigned ignore_mask, void* out, void* stream);
lsp_status lsp_shape_box(const lsp_grid* grid, int dtype, const double* lo, const double* hi,
                         unsigned ignore_mask, void* out, void* stream);
lsp_status lsp_shape_quadric(const lsp_grid* grid, int dtype, const double* center,
                             const double* weights, double offset, unsigned ignore_mask,
                             void* out, void* stream);
lsp_status lsp_shape_halfspace(const lsp_grid* grid, int dtype, const double* normal,
                               const double* point, unsigned ignore_mask, void* out,
                               void* stream);

/* Calculus on implicit functions (Sec. III-D), elementwise over n values of
 * `dtype` (device arrays; out may alias a or b):
 *  UNION       min(a, b)       interior of either
 *  INTERSECT   max(a, b)       interior of both
 *  COMPLEMENT  -a              (b unused, may be NULL)
 *  DIFFERENCE  max(a, -b)      interior of a outside b
 * Asynchronous. */
typedef enum {
    LSP_SHAPE_UNION = 0,
    LSP_SHAPE_INTERSECT = 1,
    LSP_SHAPE_COMPLEMENT = 2,
    LSP_SHAPE_DIFFERENCE = 3
} lsp_shape_op_kind;
lsp_status lsp_shape_op(int op, int dtype, const void* a, const void* b, void* out, int64_t n,
                        void* stream);

/* Wait for `stream` and report a device-side failure flagged in the
 * workspace control block since the last call that reset it (every step
 * and solve resets it on entry).  LSP_OK, LSP_ETIMEOUT (takes precedence),
 * LSP_ENONFINITE or LSP_ECUDA. */
lsp_status lsp_check_status(const void* workspace, void* stream);

/* Testing aid for the bounded waits of the persistent batched launch: from
 * now on the tiles of problem `problem` (index into the caller's arrays) are
 * never counted done, so the first wait on that problem runs out and the
 * solve reports LSP_ETIMEOUT.  -1 switches it off.  Returns the previous
 * setting.  Process-wide; not for production use. */
int lsp_debug_stall_problem(int problem);

/* Text for a status code; thread-local text of the last error. */
const char* lsp_status_string(lsp_status s);
const char* lsp_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int lsp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LSP_H */
