/*
 * les.h -- C ABI of the GB300-native time step of the DPRI urban-flow LES
 * (Vanderbauwhede, "Model Coupling between the Weather Research and
 * Forecasting Model and the DPRI Large Eddy Simulator for Urban Flows on
 * GPU-accelerated Multicore Systems", arXiv:1504.02264).
 *
 * One time step runs the paper's routines (Sec. 2.1 "LES Code Structure --
 * Functional") on one GPU:
 *   bondv1  boundary conditions: log-law inflow (standing in for the WRF
 *           wind profile of Sec. 4), zero-gradient outflow with an FP64
 *           mass-flux correction, free-slip / no-slip / periodic walls;
 *   les     Smagorinsky eddy viscosity and the SGS stress divergence;
 *   velfg   advection + diffusion "body force" (Sec. 2.5, printed u-formula);
 *   adam    second-order Adams-Bashforth on the tendency;
 *   feedbf  building forcing: zero velocity on faces touching a building;
 *   press   Poisson equation for the pressure by red-black SOR (Sec. 2.6),
 *           FP64 residual norms and stop test;
 *   velnw   projection u = u* - dt grad p, so every step ends divergence-free
 *           to the SOR tolerance.
 *
 * Conventions shared by every entry point
 *  - Return value: LES_OK (0) on success; a negative LES_E* code on error
 *    (the handle, when given, keeps a message for les_last_error); the
 *    positive status LES_ENOCONV when SOR stopped at max_sweeps above the
 *    tolerance (the step still completed and is usable).
 *  - Host arrays are owned by the caller and only read/written during the
 *    call.  Device memory is owned by the handle (allocated in les_create,
 *    released in les_destroy).
 *  - Grid: nx x ny x nz cells, i fastest.  Host array layout is C order
 *    [k][j][i].  Staggered I/O shapes: u (nz, ny, nx+1) on x-faces
 *    i = 0..nx; v (nz, ny+1, nx) on y-faces j = 0..ny; w (nz+1, ny, nx) on
 *    z-faces k = 0..nz; cell arrays p, rhs, nu_t (nz, ny, nx).  On a periodic
 *    axis face 0 and face n are the same face (equal values).
 *  - Element type of field arrays: float when grid.precision == LES_FP32,
 *    double when LES_FP64.  Norms, means and the mass flux are always FP64.
 *  - Units: metres, seconds, m/s; p is the kinematic pressure (p / rho).
 *  - A handle is not thread-safe; all its work is ordered on its stream.
 */
#ifndef LES_H
#define LES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status / error codes */
#define LES_OK 0
#define LES_ENOCONV 1        /* SOR hit max_sweeps above tol (not fatal) */
#define LES_EINVAL (-1)      /* bad argument or grid */
#define LES_ENOMEM (-2)      /* device or host allocation failed */
#define LES_ECUDA (-3)       /* a CUDA call failed (message in les_last_error) */
#define LES_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define LES_ENONFINITE (-5)  /* an FP64 norm came out NaN or Inf */
#define LES_ESTATE (-6)      /* checkpoint blob does not match this handle */

/* boundary condition per axis */
#define LES_BC_INOUT 0       /* x only: log-law inflow at x=0, outflow at x=L */
#define LES_BC_FREESLIP 1    /* y only: free-slip side walls */
#define LES_BC_WALL 2        /* z only: no-slip ground, free-slip lid */
#define LES_BC_PERIODIC 3    /* any axis; n must be even (red-black colouring) */

#define LES_FP32 0           /* FP32 fields and sweeps, FP64 norms */
#define LES_FP64 1           /* FP64 everywhere (parity / debugging) */

typedef struct les_s* les_handle;

/* Grid and step parameters; copied by les_create (dz is read during the call). */
typedef struct {
    int32_t nx, ny, nz;          /* interior cells, each >= 2 */
    int32_t bc_x, bc_y, bc_z;    /* LES_BC_* (x: INOUT|PERIODIC, y: FREESLIP|PERIODIC,
                                    z: WALL|PERIODIC) */
    double dx, dy;               /* uniform horizontal spacing (m) */
    const double* dz;            /* [nz] cell heights (m), may be stretched */
    double dt;                   /* time step (s) */
    double cs;                   /* Smagorinsky constant */
    double nu;                   /* molecular viscosity (m^2/s) */
    double omega;                /* SOR over-relaxation factor, 0 < omega < 2 */
    double tol;                  /* SOR stop: ||rhs - A p||_2 / ||rhs||_2 <= tol */
    int32_t max_sweeps;          /* SOR sweep cap per solve (one red + one black) */
    int32_t check_every;         /* residual test every this many sweeps */
    int32_t fixed_sweeps;        /* 1: always exactly max_sweeps, no stop test */
    int32_t precision;           /* LES_FP32 | LES_FP64 */
    double turb;                 /* inflow turbulence intensity (0 = laminar) */
    uint64_t seed;               /* counter-based inflow noise seed */
} les_grid_t;

/* Per-call statistics (values of the last step of the call). */
typedef struct {
    int32_t sweeps;              /* SOR sweeps in the last solve */
    int32_t status;              /* LES_OK or LES_ENOCONV */
    double rel_residual;         /* FP64 ||rhs - A p|| / ||rhs|| after the solve */
    double rhs_norm;             /* FP64 ||rhs||_2 (mean removed) */
    double rhs_mean;             /* FP64 dz-weighted fluid mean removed from rhs */
    double mass_factor;          /* outflow scaling Q_in / Q_out (1 if periodic x) */
    double q_in, q_out;          /* FP64 volume fluxes after the correction */
    double p_mean;               /* FP64 dz-weighted mean removed from p (gauge) */
    int64_t step;                /* step counter after the call */
    int64_t launches;            /* kernels launched by the handle so far */
    int32_t graph;               /* 1: the call ran its steps as CUDA graphs */
    int32_t pad_;
} les_stats_t;

/*
 * les_create: allocate device state for one domain and upload the obstacles.
 *   grid      parameters (validated: sizes >= 2, even n on periodic axes,
 *             dz > 0, 0 < omega < 2, max_sweeps >= 1, check_every >= 1).
 *   solid     [nz][ny][nx] bytes, nonzero = building cell.
 *   inflow_u  [nz] inflow speed at cell-centre heights (m/s), ignored on a
 *             periodic x axis.
 *   stream    cudaStream_t to order all work on (NULL = legacy default).
 *   out       receives the handle.
 * Initial state: all velocities, p and the Adams-Bashforth history zero,
 * step counter 0.  Returns LES_EINVAL / LES_ENOMEM / LES_ECUDA on failure
 * (no handle is returned then).
 */
int les_create(const les_grid_t* grid, const uint8_t* solid, const double* inflow_u,
               void* stream, les_handle* out);

/* les_destroy: free device memory; NULL is ignored. */
void les_destroy(les_handle h);

/* les_last_error: message of the last failing call on h (static string if h == NULL). */
const char* les_last_error(les_handle h);

/* les_set_fields: copy host u, v, w, p (I/O shapes above) into the state.
 * Keeps the Adams-Bashforth history and the step counter.  Any pointer may
 * be NULL to leave that field unchanged. */
int les_set_fields(les_handle h, const void* u, const void* v, const void* w, const void* p);

/* les_get_fields: copy the state into host buffers (NULL pointers skipped);
 * synchronises the handle's stream. */
int les_get_fields(les_handle h, void* u, void* v, void* w, void* p);

/* les_set_inflow: replace the inflow profile [nz] (m/s), intensity and seed. */
int les_set_inflow(les_handle h, const double* inflow_u, double turb, uint64_t seed);
/* les_set_inflow_series: inflow profiles that change in time (the LES side of
 * the coupling to a mesoscale model, Sec. 4, fed here by a synthetic series):
 * n profiles [n][nz] (m/s, level k fastest) at increasing times [n] (s).  Each
 * step takes at t = step * dt the linear interpolation between the two
 * bracketing profiles, held at the first / last profile outside the series;
 * the turbulence of les_set_inflow still applies on top.  n = 0 returns to
 * the fixed profile.  The series is configuration: les_get_state does not
 * store it.  Non-increasing times give LES_EINVAL. */
int les_set_inflow_series(les_handle h, int32_t n, const double* times, const double* profiles);

/*
 * les_step: advance nsteps time steps (Sec. 2.1 routine sequence, velnw last).
 * stats (nullable) receives the statistics of the last step; the call
 * synchronises the stream when stats is non-NULL or the stop test needs the
 * residual on the host.  Returns LES_ENOCONV if any step's SOR did not reach
 * tol, LES_ENONFINITE if a norm is not finite.
 */
int les_step(les_handle h, int32_t nsteps, les_stats_t* stats);

/*
 * les_pressure_solve: the press routine alone (Sec. 2.6).  rhs (nullable,
 * [nz][ny][nx], element type per precision) replaces the right-hand side
 * (non-fluid entries ignored, dz-weighted fluid mean removed); NULL reuses
 * the rhs of the last step.  Iterates red-black SOR from the current p
 * under the grid's stop rule, then removes the dz-weighted fluid mean of p.
 */
int les_pressure_solve(les_handle h, const void* rhs, les_stats_t* stats);

/* Intermediate arrays for inspection (copied to host, synchronising). */
#define LES_AUX_NUT 0        /* nu_t (nz, ny, nx) of the last step */
#define LES_AUX_RHS 1        /* Poisson rhs (nz, ny, nx), mean removed */
#define LES_AUX_USTAR 2      /* u* (nz, ny, nx+1) of the last step */
#define LES_AUX_VSTAR 3      /* v* (nz, ny+1, nx) */
#define LES_AUX_WSTAR 4      /* w* (nz+1, ny, nx) */
#define LES_AUX_FU 5         /* Adams-Bashforth history F_u (u shape) */
#define LES_AUX_FV 6
#define LES_AUX_FW 7
#define LES_AUX_R0 8         /* initial residual rhs - mean - A p_prev of the last solve (recording on) */
#define LES_AUX_DELTA 9      /* correction p_solved - p_prev of the last solve, before the gauge (recording on) */
#define LES_AUX_MASK 10      /* 1 on Poisson unknowns (fluid cells with an open face), else 0 */
#define LES_AUX_NET_IN 11    /* residual (nz, ny, nx) the learned start-of-solve correction of the last
                                solve that ran one took as the network input (recording on; FP32 grids) */
#define LES_AUX_NET_Q 12     /* that correction's network prediction q (nz, ny, nx), 0 off the unknowns */
/* LES_AUX_R0 / DELTA / NET_IN / NET_Q need recording on (LES_EINVAL otherwise)
 * and a solve that recorded them (LES_ESTATE otherwise). */
int les_get_aux(les_handle h, int32_t which, void* out);

/* les_set_record: keep the initial residual and the total correction of every
 * solve (LES_AUX_R0 / LES_AUX_DELTA), the training pairs of the warm-start
 * network.  Costs two device copies per solve while on. */
int les_set_record(les_handle h, int32_t enable);
/* les_set_record_at: take the recorded pair at the first FP64 refinement at
 * or after `after_sweeps` sweeps instead of at the start of the solve: the
 * residual r_k of the iterate p_k there and the remaining correction
 * p_solved - p_k (the pairs a network applied inside the solve sees).
 * 0 = at the start (default).  A value > 0 runs solves from the host loop.
 * A solve that passes the stop test before the record point records no
 * pair: LES_AUX_R0 / LES_AUX_DELTA then return LES_ESTATE until one does. */
int les_set_record_at(les_handle h, int32_t after_sweeps);

/*
 * Checkpoint / restart: the full state (velocities, p, AB2 history, step
 * counter, inflow profile and noise seed) as an opaque blob.  les_get_state
 * with buf == NULL stores the required size in *len; otherwise *len must be
 * at least that size.  les_set_state accepts only a blob of a handle with the
 * same grid (else LES_ESTATE).  A restored handle continues bit-identically.
 */
int les_get_state(les_handle h, void* buf, size_t* len);
int les_set_state(les_handle h, const void* buf, size_t len);

/*
 * Phase timing with CUDA events recorded on the handle's stream (the
 * per-routine breakdown the paper reports for its kernels, Sec. 2.7).
 * les_set_timing(h, 1) zeroes and enables the accumulators; 0 disables.
 * Enabled timing adds one stream synchronisation per step.
 */
typedef struct {
    double ms_momentum;          /* bondv1 + les + velfg + adam + feedbf + rhs */
    double ms_sor;               /* SOR sweep kernels only */
    double ms_residual;          /* FP64 residual / stop-test kernels */
    double ms_project;           /* velnw (projection + gauge) */
    int64_t steps;               /* steps timed */
    int64_t sor_sweeps;          /* SOR sweeps timed */
    int64_t sor_launches;        /* SOR kernel launches timed */
    int64_t launches;            /* all kernels launched by the handle so far */
    double ms_net;               /* learned correction: prediction, line search, step */
    int64_t net_cycles;          /* learned corrections timed inside the solve loop */
} les_timing_t;
int les_set_timing(les_handle h, int32_t enable);
int les_get_timing(les_handle h, les_timing_t* t);

/*
 * Step execution mode.  enable = 1 (default): the solve loop runs as
 * captured CUDA graphs of several batches of sweeps each (estimate and
 * refinement included); every kernel in them returns at once when the
 * device-side stop test has set its flag, and the host reads a mapped copy
 * of the flag one graph behind (with fixed_sweeps the whole step is one
 * graph).  enable = 0: host-driven loop, reading the residual back after
 * every batch of check_every sweeps.  Phase timing (les_set_timing) always uses the
 * host-driven loop.  Both modes compute the same iterates.
 */
int les_set_graph(les_handle h, int32_t enable);

/*
 * SOR sweep kernel selection.  tile = -1 runs the two in-place half-sweep
 * kernels; tile = 0..LES_SOR_NTILES-1 runs a fused red-black kernel: tiles
 * whose les_sor_tile tz is 0 are column tiles marching kc planes per CTA
 * (kc <= 0: the whole column), the others are tx x ty x tz blocks (kc
 * ignored); tiles 17-24 are 28 x ty x tz blocks loaded by the tensor-memory
 * accelerator (FP32 grids only, else LES_EINVAL), 21-24 in persistent CTAs
 * that prefetch their next block (FP32 grids without periodic axes only,
 * else LES_EINVAL); tiles 25-28 are 30 x ty columns that march through kc
 * planes per CTA with a pipeline of per-plane TMA copies (FP32 grids, any
 * boundary conditions; kc <= 0 picks the chunk that gives at least two CTAs
 * per SM); tiles 29-34 are 28 x ty x tz TMA blocks whose lanes walk columns of
 * one colour up the block (FP32 grids, any boundary conditions).
 * Every choice computes the same iterate.
 * les_autotune_sor times each tile shape with a few k-chunk lengths on this
 * handle's grid (sweeps per candidate), keeps the fastest and reports it;
 * the field state is saved and restored around the trial sweeps.
 */
#define LES_SOR_NTILES 35
int les_set_sor_config(les_handle h, int32_t tile, int32_t kc);
int les_get_sor_config(les_handle h, int32_t* tile, int32_t* kc);
int les_sor_tile(int32_t tile, int32_t* tx, int32_t* ty, int32_t* tz);
int les_autotune_sor(les_handle h, int32_t sweeps, double* best_ms_per_sweep);
/* les_time_sor: milliseconds per sweep of one configuration (tile index of
 * les_set_sor_config, kc) timed over `sweeps` sweeps on the scratch
 * correction buffers (state untouched, configuration kept).  LES_EINVAL for
 * a tile this grid cannot use. */
int les_time_sor(les_handle h, int32_t tile, int32_t kc, int32_t sweeps, double* ms_per_sweep);

/*
 * les_sor_compare: the solver's red-black SOR next to the paper's "twinned
 * double buffering" (Sec. 2.6) on one pressure problem.  From p0, run
 * `sweeps` sweeps of the variant on the correction equation A d = rhs - A p0
 * (FP64 residual, sweeps in the handle's field type) and report:
 *   p_out        p0 + d (host, dense nx*ny*nz FP64, i fastest; nullable);
 *   ms_per_sweep device time per sweep (CUDA events on the handle's stream);
 *   rel_residual FP64 ||rhs - A (p0 + d)|| / ||rhs|| over the unknowns.
 * Variants:
 *   LES_SOR_REDBLACK  the update printed in Sec. 2.6, red cells (i+j+k odd)
 *                     then black, with this handle's sweep kernel and tile;
 *   LES_SOR_TWINNED   two copies of the correction interleaved as pairs
 *                     (the paper's array of two-float vectors): for nrd = 0
 *                     copy 1 takes the printed update of every unknown with
 *                     all neighbours from copy 0, for nrd = 1 copy 0 from
 *                     copy 1.  This is a weighted Jacobi iteration: it
 *                     converges for 0 < omega < 1 on these operators and
 *                     diverges at the SOR value 1.7.
 * omega > 0 overrides the grid's relaxation factor for the call; omega <= 0
 * keeps it.  rhs and p0: host, dense nx*ny*nz FP64; rhs must be compatible
 * (zero dz-weighted mean over the fluid cells) for the residual to fall.
 * The handle's state is untouched (scratch buffers are allocated on first
 * use and kept); sweeps >= 1.  LES_EINVAL for a bad variant or argument.
 */
#define LES_SOR_REDBLACK 0
#define LES_SOR_TWINNED 1
int les_sor_compare(les_handle h, int32_t variant, double omega, int32_t sweeps, const double* rhs,
                    const double* p0, double* p_out, double* ms_per_sweep, double* rel_residual);

/*
 * les_residual_noalloc: FP64 norms of the pressure Poisson residual for
 * callers that cannot allocate device memory (code running inside another
 * framework's memory pool, programs with a device-memory budget fixed at
 * start-up, or callers that must not allocate while a stream capture is in
 * progress elsewhere).  The paper has no counterpart: this is a service entry
 * point next to the handle API, and it allocates nothing.
 *
 *   grid     nx, ny, nz, bc_x/y/z, dx, dy and precision are read (dz, the
 *            SOR settings and the rest are ignored).
 *   d_p      device array (nz, ny, nx) of pressure, element type per
 *            precision (float for LES_FP32, double for LES_FP64).
 *   d_rhs    device array (nz, ny, nx), same type: the right-hand side as is
 *            (no mean is removed).
 *   d_solid  device array (nz, ny, nx) of bytes, nonzero = building cell.
 *   d_dz     device array [nz] of cell heights (double).
 *   d_out    device array of 3 doubles written on completion:
 *            [0] sum r^2, [1] sum rhs^2, [2] sqrt([0]/[1]) (sqrt([0]) when
 *            [1] == 0), with r = rhs - A p over the fluid cells that have an
 *            open face, A the operator of les_pressure_solve.
 *   stream   cudaStream_t the work is ordered on (NULL = legacy default).
 * The caller owns every buffer.  The only scratch is a fixed device array of
 * about 64 KB in this library (4096 FP64 partial-sum pairs and a counter);
 * the entry point never calls cudaMalloc, cudaFree or any allocating routine.
 * The array is placed on a device when the library's module loads there:
 * with CUDA's default lazy module loading that is the first call of this
 * entry point on the device, so callers on a fixed device-memory budget make
 * one call at start-up (or set CUDA_MODULE_LOADING=EAGER); it then stays
 * resident on that GPU until the process exits.  On its first call on a
 * device (with that device current), and again whenever the device's current
 * context has changed (after a device reset, say), it looks up the array's
 * device address; make that first call before any stream capture.  Each call
 * clears the counter before use.  All calls share the array, so calls whose
 * kernels overlap on the GPU (different streams, or different host threads)
 * race and give wrong norms: order them.  Grids above LES_NOALLOC_MAX_CELLS
 * cells (a chosen bound; grids of any size below it run with at most 4096
 * blocks striding over the cells) and bad arguments give LES_EINVAL; CUDA
 * failures LES_ECUDA.  Asynchronous: read d_out after synchronising the
 * stream.
 */
#define LES_NOALLOC_MAX_CELLS 2147483647LL
int les_residual_noalloc(const les_grid_t* grid, const void* d_p, const void* d_rhs, const uint8_t* d_solid,
                         const double* d_dz, double* d_out, void* stream);

/*
 * Learned SOR warm start (no counterpart in the paper, which warm-starts SOR
 * from the previous step's pressure).  A 4-level 3-D U-Net (3x3x3 convs,
 * 16/32/64/128 channels, bias-free, ReLU, 2x2x2 mean pooling, nearest
 * upsampling, additive skips, 1x1x1 head) maps the solve's initial residual
 * r0 = rhs - mean - A p_prev (scaled to unit RMS) and the unknown mask to a
 * correction direction q.  The solver then takes p0 = p_prev + alpha q with
 * alpha = <q, V r0> / <q, V A q> in FP64 (V = diag(dz_k); V A is symmetric),
 * the minimiser of the energy norm of the error along q, so p0 is never
 * further from the solution than p_prev in that norm, and runs the same
 * red-black SOR to the same tolerance: plain SOR stays the stop test.  Activations are BF16, accumulation FP32, on the
 * tensor cores: the forward convolutions (and the backward pass's input
 * gradients) on tcgen05.mma with the accumulator in tensor memory by default,
 * or on the warp-level mma.sync kernel (les_net_set_engine); the weight
 * gradients on mma.sync.  Training runs on the GPU with the network's own
 * backward kernels and Adam.
 *
 * Device arrays of the training / inference calls are dense float [b][nz][ny][nx]
 * (b = batch index): d_r residuals, d_mask 1/0 unknown masks, d_t target
 * corrections; the loss is the batch mean of mean_mask (y - t / rms_mask(t))^2.
 * les_net_gradient writes the flat FP32 gradient (les_net_num_params floats:
 * conv0..conv6 as [27][Cout][Cin], tap = (dz*3+dy)*3+dx, then the 16 head
 * weights) without updating; les_net_train_step applies Adam (beta 0.9/0.999).
 */
typedef struct les_net_s* les_net;
#define LES_WARM_PREV 0      /* p0 = p from the previous step (the paper's scheme) */
#define LES_WARM_NET 1       /* p0 = p_prev + alpha * network(r0) */
#define LES_WARM_ZERO 2      /* p0 = 0 (cold start every step; a reference point for the two above) */
int les_net_create(uint64_t seed, void* stream, les_net* out);
void les_net_destroy(les_net n);
const char* les_net_last_error(les_net n);
int les_net_num_params(les_net n, int64_t* count);
int les_net_get_params(les_net n, float* host);
int les_net_set_params(les_net n, const float* host);
/* les_net_set_stride: run the network on the grid coarsened `stride` times per
 * axis (1, 2, 4 or 8; default 1).  Inputs are pooled (block sums / stride^3,
 * cells outside the grid count as zero: the pooled mask is the unknown
 * fraction), the network runs at the coarse level and its output is
 * prolongated to the fine cells by trilinear interpolation between coarse
 * cell centres (clamped at the boundary) and masked: a learned coarse-grid
 * correction.  Training calls take fine arrays and train at the coarse level
 * against the pooled target. */
int les_net_set_stride(les_net n, int32_t stride);
int les_net_get_stride(les_net n, int32_t* stride);
/* les_net_set_engine: the tensor-core path of the forward convolutions:
 * LES_NET_TCGEN05 (default: tcgen05.mma, 128-voxel x 16/32-channel tiles,
 * FP32 accumulator in tensor memory) or LES_NET_MMA_SYNC (warp-level
 * m16n8k16).  Both stage the same BF16 operands and accumulate in FP32 (the
 * summation order inside an MMA differs).  With LES_NET_TCGEN05 the CTAs
 * that split a small layer's input channels form a thread-block cluster and
 * add their partial sums over distributed shared memory (where the device
 * can co-schedule such clusters); LES_NET_TCGEN05_GMEM_SPLIT adds them
 * through global memory instead, with the same sums in the same order
 * (bit-identical results).  A tcgen05 kernel whose bounded wait gives up
 * makes the next synchronous network call return LES_ETIMEOUT. */
#define LES_NET_MMA_SYNC 0
#define LES_NET_TCGEN05 1
#define LES_NET_TCGEN05_GMEM_SPLIT 2
int les_net_set_engine(les_net n, int32_t engine);
int les_net_get_engine(les_net n, int32_t* engine);
int les_net_forward(les_net n, const float* d_r, const float* d_mask, float* d_y, int32_t nx, int32_t ny, int32_t nz);
int les_net_gradient(les_net n, const float* d_r, const float* d_mask, const float* d_t, int32_t batch, int32_t nx,
                     int32_t ny, int32_t nz, float* d_grad, double* loss);
int les_net_train_step(les_net n, const float* d_r, const float* d_mask, const float* d_t, int32_t batch, int32_t nx,
                       int32_t ny, int32_t nz, float lr, double* loss);
/* les_set_warmstart: LES_WARM_NET needs an FP32 grid; the handle keeps the
 * network pointer (the caller keeps it alive). */
int les_set_warmstart(les_handle h, int32_t mode, les_net net);
/* les_set_net_schedule: with LES_WARM_NET, also apply the network inside the
 * solve every `every_sweeps` sweeps (at an FP64 refinement: q = Net(r_k),
 * p += alpha q with the energy-norm step, residual formed again), i.e. the
 * network as a coarse correction between SOR batches.  0 = only at the
 * start (default).  A value > 0 runs solves from the host loop.  The stop
 * test is unchanged. */
int les_set_net_schedule(les_handle h, int32_t every_sweeps);
/* les_set_net_kernels: how the kernels of a network correction are laid out.
 * LES_NET_KERNELS_FOLDED (0, default, fastest inside the CUDA graphs on
 * GB300): one launch per layer, with the packing of the network input run
 * inside the first convolution's staging and the head inside the last
 * convolution's epilogue (tcgen05 engine), and the trilinear prolongation
 * inside the line search, which prolongs the coarse output on the fly.
 * LES_NET_KERNELS_LAYERS (2): the same layers with the packing, head and
 * prolongation as kernels of their own; it computes the same values as 0
 * (bit-identical fields) and serves to check the folded kernels.
 * LES_NET_KERNELS_PERSISTENT (1): the coarse network (RMS, packing, the
 * seven convolutions, head) as one cooperative persistent launch with a
 * bounded grid barrier between layers, when the device supports cooperative
 * launches; the same correction up to the summation order of the RMS.
 * With 0 or 2 on an FP32 grid with no periodic axis, at network stride 4 or
 * 8 and the in-place schedule, the estimate after each batch of sweeps also
 * pools the residual and the unknown mask over the stride cubes and forms
 * their RMS, and the correction skips its pooling kernel; or-ing
 * LES_NET_KERNELS_OWN_POOL (4) into the mode keeps the pooling kernel (the
 * same pooled input up to the FP32 summation order of each cube).
 * Any other value: LES_EINVAL. */
#define LES_NET_KERNELS_FOLDED 0
#define LES_NET_KERNELS_PERSISTENT 1
#define LES_NET_KERNELS_LAYERS 2
#define LES_NET_KERNELS_OWN_POOL 4
int les_set_net_kernels(les_handle h, int32_t mode);
/* les_set_net_async: with a schedule (every_sweeps > 0) in the CUDA-graph
 * loop, 1 overlaps each network prediction with the next batch of sweeps:
 * the prediction made from the residual of batch b runs on a second stream
 * while batch b+1 sweeps, and is applied after it (the energy-norm step
 * against the then current residual, which becomes the residual of the
 * corrected iterate and the next prediction's input).  The step can never
 * raise the error's energy, and the stop test is unchanged; the sweep count
 * can differ from the in-place correction.  The host-driven loop (timing,
 * recording) keeps the in-place correction.  Default 0. */
int les_set_net_async(les_handle h, int32_t enable);
/* les_set_net_start: with a schedule (every_sweeps > 0), whether the network
 * also corrects p at the start of each solve (default 1); without a schedule
 * the start correction is the warm start and always runs. */
int les_set_net_start(les_handle h, int32_t enable);

/*
 * Ensembles: n domains of uneven size, each with its own buildings, inflow
 * and state, stepped together.  Every member is an ordinary FP32 domain
 * handle created from grids[i], solid[i], inflow[i] exactly as by
 * les_create, on the ensemble's stream; les_ensemble_member gives the
 * handle for les_set_fields / les_get_fields / les_get_aux / les_get_state
 * (the ensemble owns it: do not destroy it, and step members only through
 * les_ensemble_step, else the next ensemble step returns LES_ESTATE).
 * The SOR solves of all members run as batched launches over a flattened
 * (member, tile) work list: one persistent sweep launch per sweep for the
 * whole ensemble (28 x BY x BZ row tiles, `tile` 0..4 = 8x8, 4x8, 8x4,
 * 16x4, 4x16; ctas_per_sm CTAs per SM walk the list) -- or, with `tile` 5,
 * one launch per member per sweep with the member's own kernel and tile
 * (les_set_sor_config / les_autotune_sor of the member; TMA where its grid
 * allows) -- or, with `tile` 6, one persistent launch per sweep whose CTAs
 * walk every member's 28 x 8 x 8 blocks with that member's tensor maps (the
 * TMA block kernel of tile 17, ctas_per_sm ignored) -- one estimate and one
 * refinement launch per batch of check_every sweeps, chunks of batches in
 * CUDA graphs; each member stops at its own tolerance and sweep count.  A
 * member evolves bit-identically to the same domain stepped alone with the
 * same row tile (les_set_sor_config(h, 12 + tile, 0)), or with tile 17 in
 * the batched TMA mode.
 * Requirements (else LES_EINVAL): 1 <= n <= 64; every member FP32, tolerance
 * mode (fixed_sweeps = 0), the same even check_every, and max_sweeps a
 * multiple of it.  The ensemble keeps no pointer to the caller's arrays.
 * les_ensemble_step fills stats[i] for member i after the last step when
 * stats is not NULL (n entries); returns LES_ENOCONV if any member ended
 * above its tolerance.  les_ensemble_autotune times `sweeps` batched sweeps
 * per (tile, CTAs per SM) candidate and the per-member mode (after
 * autotuning every member) on the members' scratch correction buffers (the
 * state is not changed) and keeps the fastest.
 */
typedef struct les_ensemble_s* les_ensemble;
int les_ensemble_create(int32_t n, const les_grid_t* grids, const uint8_t* const* solid, const double* const* inflow,
                        void* stream, les_ensemble* out);
void les_ensemble_destroy(les_ensemble e);
const char* les_ensemble_last_error(les_ensemble e);
int les_ensemble_size(les_ensemble e, int32_t* n);
int les_ensemble_member(les_ensemble e, int32_t i, les_handle* out);
int les_ensemble_step(les_ensemble e, int32_t nsteps, les_stats_t* stats);
int les_ensemble_set_graph(les_ensemble e, int32_t enable);
int les_ensemble_set_tile(les_ensemble e, int32_t tile, int32_t ctas_per_sm);
int les_ensemble_get_tile(les_ensemble e, int32_t* tile, int32_t* ctas);
int les_ensemble_autotune(les_ensemble e, int32_t sweeps, double* best_ms_per_sweep);
int les_ensemble_launches(les_ensemble e, int64_t* launches);
/* les_ensemble_set_persistent: 1 runs the SOR solve of every plain-SOR step
 * (no network set with les_ensemble_set_warmstart) as one persistent
 * cooperative launch per step: its CTAs walk, batch after batch, every
 * running member's TMA blocks for each sweep, then the estimates, the FP64
 * accumulations and residuals with their stop decisions, separated by a
 * bounded grid barrier, until every member's solve has ended; the launches
 * of a step do not depend on its sweeps.  Selects the batched TMA mode
 * (tile 6, whose arithmetic it shares bit for bit).  With a network the
 * ensemble keeps its chunk graphs.  LES_EINVAL if the device cannot run a
 * cooperative launch; a grid barrier that times out makes the step return
 * LES_ETIMEOUT.  0 (default) returns to the chunk graphs. */
int les_ensemble_set_persistent(les_ensemble e, int32_t enable);
/* les_ensemble_set_warmstart: every member applies the learned correction
 * `net` at the start of its solve and every `every_sweeps` sweeps inside it
 * (even, dividing each member's max_sweeps; the batch size of the ensemble's
 * loop becomes every_sweeps); net = NULL returns to the previous-step start.
 * The members share the network (its workspace is sized for the largest). */
int les_ensemble_set_warmstart(les_ensemble e, les_net net, int32_t every_sweeps);

/* Failure-detection self-test: launches one block whose bounded device wait
 * (the one the TMA sweeps use: an mbarrier polled against the global timer)
 * waits for a transaction that never arrives.  It must give up after
 * limit_ns (1e3..2e9) and report it: returns LES_ETIMEOUT (the expected
 * result; les_last_error(NULL) says so), LES_OK if the wait completed,
 * LES_ECUDA/LES_ENOMEM on CUDA errors.  Nothing is left in flight; the CUDA
 * context stays usable. */
int les_selftest_wait_timeout(int64_t limit_ns, void* stream);

/* Bracket a region for a profiler started with capture off
 * (cudaProfilerStart when start != 0, cudaProfilerStop otherwise). */
int les_profiler_range(int32_t start);

/* Library version string. */
const char* les_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LES_H */
