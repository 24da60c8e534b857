/*
 * lb.h - C ABI of the GB300 (sm_103a) hybrid thermal pseudopotential lattice
 * Boltzmann boiling step (Li, Kang, Francois, He, Luo; arXiv 1501.03857).
 *
 * One time step advances the D2Q9 MRT populations with the improved forcing
 * scheme (Eqs. 2-9), the Peng-Robinson pseudopotential (Eq. 21) and the
 * wettability force (Eq. 22), integrates the temperature equation (Eq. 18)
 * with classical RK4 (Eqs. 19-20) and isotropic central differences, and
 * accumulates the bottom-wall heat flux q(t) (Sec. 3.2).
 *
 * Conventions shared by every entry point
 *  - Every call returns LB_OK (0) or a negative LB_E_* code; the message of
 *    the last failure on the calling thread is returned by lb_last_error().
 *    Nothing aborts, traps or prints.
 *  - Fields are row-major [y][x] with x fastest, rows y = 0 (heated bottom
 *    wall) .. Ly-1 (top). Populations are [alpha][y][x] with the velocity
 *    order e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1)
 *    e7=(-1,-1) e8=(1,-1).
 *  - Units are lattice units (delta_x = delta_t = 1, Sec. 3.1).
 *  - The caller owns every device buffer (the workspace) and the CUDA stream
 *    (passed as void*, a cudaStream_t). The handle owns host metadata only.
 *    All device work is issued asynchronously on that stream; entry points
 *    that return host data synchronise the stream first.
 *  - Device-detected faults (EOS domain, non-finite values) latch a flag
 *    that the next synchronising call (lb_sync, lb_heat_flux, lb_fields,
 *    lb_get_state, lb_mass) reports as LB_E_EOS_DOMAIN / LB_E_NONFINITE and
 *    then clears; in the bounds-checked build (liblbboil_checked.so) an
 *    address outside its buffer is reported the same way as LB_E_BOUNDS.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_OK 0
#define LB_E_INVAL (-1)       /* bad argument, size or state                */
#define LB_E_CUDA (-2)        /* a CUDA runtime call failed                 */
#define LB_E_EOS_DOMAIN (-3)  /* psi argument 2(p - rho/3)/G < 0 somewhere  */
#define LB_E_NONFINITE (-4)   /* NaN or Inf in rho or T                     */
#define LB_E_TIMEOUT (-5)     /* a bounded device wait gave up              */
#define LB_E_BOUNDS (-6)      /* checked build only: a device index left its
                                 buffer (the access was skipped)            */

/* Boundary condition in y (Sec. 3.1: periodic in x, solid walls at y = 0
 * and y = Ly). */
#define LB_BC_WALLS 0         /* Zou-He no-slip walls, T_b below, T_s above */
#define LB_BC_TOP_OUTFLOW 1   /* bottom wall; top row zero-gradient, T_s    */
#define LB_BC_PERIODIC 2      /* periodic in y too (invariant tests)        */

/* Grid and switches. Lx >= 1, Ly >= 3. */
typedef struct lb_grid {
    int32_t Lx, Ly;
    int32_t bc_y;         /* LB_BC_*                                         */
    int32_t ghost_layer;  /* 1: apply F_m on wall rows with a ghost row that
                             copies the wall row's psi (Sec. 3.2's ghost-
                             layer variant, for which the paper reports
                             about 90 degrees; with this reading a droplet
                             at G_w = 0 settles near 138 degrees);
                             0: no F on wall rows (about 44.5 degrees)       */
    int32_t isothermal;   /* 1: skip the temperature equation (T frozen)     */
    int32_t reserved;
} lb_grid;

/* Peng-Robinson EOS (Eq. 21) and pseudopotential parameters. The paper
 * uses a = 3/49, b = 2/21, R = 1, omega = 0.344, sigma = 1.2 (after Eq. 21);
 * G must be negative (psi = sqrt(2 (p - rho c_s^2)/(G c^2)), after Eq. 7). */
typedef struct lb_eos {
    double a, b, R, omega, G, sigma;
} lb_eos;

/* Thermal and transport parameters (Sec. 3.1) and the initial pool.
 * Paper values: T_s = 0.86 T_c, c_v = 6, c_v chi = 0.028, g = 3e-5,
 * nu_L = 0.1, nu_V = 0.5/3. s_e, s_zeta, s_q are the relaxation rates of
 * Eq. 4 that the paper leaves unstated (defaults 0.8, 0.8, 1.1). The
 * initial state is liquid below y = pool_height and vapour above with a
 * tanh interface of width 5 and relative density noise +-noise_amp drawn
 * from splitmix64(seed, y*Lx + x). */
typedef struct lb_thermal {
    double Ts_over_Tc, cv, cv_chi, g, nu_l, nu_v, s_e, s_zeta, s_q;
    double pool_height, noise_amp;
    uint64_t seed;
} lb_thermal;

typedef struct lb_handle lb_handle;

/* ---- host-only helpers (no GPU needed) -------------------------------- */

/* T_c = 0.0778 a / (0.45724 b R), from the two relations after Eq. 21. */
int lb_critical_temperature(const lb_eos* eos, double* Tc);

/* Maxwell equal-area coexistence densities of the PR EOS at temperature T
 * (0 < T < T_c), solved in FP64 on the host (Sec. 3.1: rho_L ~ 6.5 and
 * rho_V ~ 0.38 at 0.86 T_c). */
int lb_coexistence(const lb_eos* eos, double T, double* rho_v, double* rho_l);

/* The initial density lb_init builds when rho0 == NULL (Sec. 3.1 set-up),
 * written to the caller's host array rho0[Ly*Lx]. */
int lb_initial_density(const lb_grid* grid, const lb_eos* eos,
                       const lb_thermal* th, float* rho0);

/* Device workspace bytes lb_init needs for this grid (populations and
 * temperature, double-buffered, plus accumulators). Population offsets are
 * 32-bit: grids with 9 * pitch * Ly >= 2^31 (pitch = Lx rounded up to a
 * multiple of 32; e.g. Ly > 14563 at Lx = 16384) are rejected with
 * LB_E_INVAL, here and by lb_init. */
int lb_workspace_bytes(const lb_grid* grid, size_t* bytes);

/* ---- simulation --------------------------------------------------------- */

/* Create a simulation in the caller's device workspace (>= the size from
 * lb_workspace_bytes, 256-byte aligned) on stream `stream` (a cudaStream_t).
 * Tb_profile: NULL or Lx values added to `superheat` to give the bottom-wall
 * superheat T_b(x) - T_s (Sec. 3.2 defines Delta T = T_b - T_s). Gw: the
 * fluid-solid interaction strength of Eq. 22 on the heating wall. rho0: NULL
 * (build the pool from `th`) or a host array [Ly*Lx] of initial densities.
 * The populations start at the rest equilibrium w_a rho0 and T = T_s, with
 * the wall rows at their Dirichlet temperatures. rho_ave of Eq. 9 is the
 * mean of rho0. Synchronises the stream before returning. */
int lb_init(lb_handle** h, const lb_grid* grid, const lb_eos* eos,
            const lb_thermal* th, const double* Tb_profile, double superheat,
            double Gw, const float* rho0, void* dev_workspace,
            size_t workspace_bytes, void* stream);

/* Advance nsteps (>= 0) time steps asynchronously on the stream; each step
 * adds one sample q(t) (level t, before the step's update) to the device
 * FP64 heat-flux accumulators. */
int lb_step(lb_handle* h, int nsteps);

/* Change the bottom-wall temperature (the superheat step of Sec. 3.2):
 * T_b(x) - T_s = superheat + (Tb_profile ? Tb_profile[x] : 0). Takes effect
 * at the next step (the current wall row is overwritten too). Asynchronous;
 * Tb_profile may be reused as soon as the call returns. */
int lb_set_wall_temperature(lb_handle* h, const double* Tb_profile, double superheat);

/* Change G_w of Eq. 22. */
int lb_set_wettability(lb_handle* h, double Gw);

/* Read the wall heat-flux statistics (Sec. 3.2): q_inst = the last q(t),
 * q_mean and q_std over the samples since the last reset, nsamples. Any
 * output pointer may be NULL. reset != 0 clears the sums after reading.
 * Synchronises the stream. */
int lb_heat_flux(lb_handle* h, double* q_inst, double* q_mean, double* q_std,
                 int64_t* nsamples, int reset);

/* Macroscopic fields at the current time level: rho = sum f, u = (sum e f
 * + F/2)/rho with the forces of this level (Eq. 6), T = T_s + theta. Each
 * output is [Ly*Lx] FP32 or NULL; on_device != 0 means device pointers.
 * Synchronises the stream. */
int lb_fields(lb_handle* h, float* rho, float* ux, float* uy, float* T, int on_device);

/* Copy the raw state out / in: post-collision populations fpost[9*Ly*Lx]
 * and theta = T - T_s [Ly*Lx] (either may be NULL). lb_get_state
 * synchronises; lb_set_state is asynchronous (the source must stay valid
 * until the stream reaches it when on_device != 0). */
int lb_get_state(lb_handle* h, float* fpost, float* theta, int on_device);
int lb_set_state(lb_handle* h, const float* fpost, const float* theta, int on_device);

/* Total mass sum_x rho = sum_x sum_a f*_a, accumulated in FP64 on the
 * device (Eq. 9's rho_ave is mass / (Lx Ly) at t = 0). Synchronises. */
int lb_mass(lb_handle* h, double* mass);

/* Wait for the stream and report latched device faults. */
int lb_sync(lb_handle* h);

/* Number of steps taken, and the launch shape in use: threads per block
 * (a multiple of 32; 10 of them are x-halo columns) and rows per segment. */
int lb_info(lb_handle* h, int64_t* steps, int* block_x, int* seg_rows, int* nblocks);

/* Override the launch shape of the fused step (seg_rows >= 1; 0 keeps the
 * automatic choice; block_x 64, 128 or 256, 0 for the default: 64 up to
 * 4096 columns, 128 beyond). Results do not depend on the launch shape.
 * Used by the autotuner. */
int lb_set_launch(lb_handle* h, int block_x, int seg_rows);

/* Checkpoint: lb_save_bytes gives the blob size; lb_save writes the state,
 * step count, accumulators and wall profile into host memory; lb_load
 * restores a blob saved from a handle with the same grid. Both
 * synchronise. */
int lb_save_bytes(lb_handle* h, size_t* bytes);
int lb_save(lb_handle* h, void* host_buf, size_t bytes);
int lb_load(lb_handle* h, const void* host_buf, size_t bytes);

/* Release the handle (the workspace stays the caller's). */
int lb_destroy(lb_handle* h);

/* ---- gradients (discrete adjoint) ----------------------------------------- */

/* Device scratch lb_adjoint needs for nsteps steps with a checkpoint every
 * ckpt_every steps (work fields, checkpoints, two replayed segments with the
 * forward intermediates of their steps: about 10 nsteps / ckpt_every + 40
 * ckpt_every planes of Lx * Ly floats; with ckpt_every = 1, every step's
 * state and intermediates: about 20 nsteps planes). */
int lb_adjoint_scratch_bytes(lb_handle* h, int nsteps, int ckpt_every, size_t* bytes);

/* Checkpoint interval for lb_adjoint over nsteps steps whose scratch fits in
 * budget_bytes of device memory. 1 (every step's state and intermediates
 * stored, no replay: the fastest) when its scratch fits; otherwise the
 * interval with the smallest scratch (checkpoints take ~10 nsteps / C
 * planes and the replay buffers ~40 C, so about C = sqrt(nsteps / 4)), whose
 * run time is about the same for every C >= 2 (each step is replayed once).
 * Writes the interval to *ckpt_every and, if bytes is not NULL, its scratch
 * to *bytes (as lb_adjoint_scratch_bytes). LB_E_INVAL when no interval fits
 * (nothing written), for a null output, or when lb_adjoint would reject the
 * run. Host arithmetic only; nothing is issued on the stream. */
int lb_adjoint_pick_ckpt(lb_handle* h, int nsteps, size_t budget_bytes, int* ckpt_every, size_t* bytes);

/* Gradient of the window-averaged bottom-wall heat flux
 * J = (1/nsteps) sum_{n} q(t_n) over the next nsteps steps (Sec. 3.2) with
 * respect to the bottom-wall temperature profile T_b(x) (dJ_dTb, host [Lx])
 * and the wettability strength G_w of Eq. 22 (dJ_dGw, host), by the discrete
 * adjoint (reverse mode) of the step. The state at the window start is held
 * fixed except its bottom wall row, which is T_b. Runs the nsteps forward
 * steps (the simulation advances; its heat-flux accumulators are not
 * touched) storing a checkpoint every ckpt_every steps, then sweeps back,
 * replaying each segment from its checkpoint. With ckpt_every = 1 the
 * forward steps store every step's state and forward intermediates and the
 * sweep replays nothing: faster, for ~20 planes of scratch per step. J
 * (host) receives the value.
 * Walls or the outflow top in y, with or without the ghost layer, thermal runs
 * only. A fault met by the window's forward steps is returned as
 * LB_E_EOS_DOMAIN or LB_E_NONFINITE (LB_E_BOUNDS in the checked build), with
 * the simulation's own fault flags left clear; the simulation has then been
 * advanced through the window all the same.
 * Synchronises. */
int lb_adjoint(lb_handle* h, int nsteps, int ckpt_every, void* dev_scratch, size_t scratch_bytes,
               double* J, double* dJ_dTb, double* dJ_dGw);

/* ---- batches: many independent simulations, one launch per step ---------- */

/* One instance of a batch (the points of a boiling curve, Sec. 3.2-3.3:
 * superheat x wettability): its grid, parameters, bottom-wall superheat
 * T_b(x) - T_s = superheat + (Tb_profile ? Tb_profile[x] : 0) (host, may be
 * NULL), G_w of Eq. 22, and an optional host initial density rho0[Ly*Lx]
 * (NULL: the pool of th). */
typedef struct lb_batch_desc {
    lb_grid grid;
    lb_eos eos;
    lb_thermal th;
    double superheat, Gw;
    const double* Tb_profile;
    const float* rho0;
} lb_batch_desc;

typedef struct lb_batch lb_batch;

/* Device workspace for n instances (each laid out as for lb_init, plus the
 * per-step parameter tables). */
int lb_batch_workspace_bytes(const lb_batch_desc* d, int n, size_t* bytes);

/* Create n instances in one caller workspace on `stream`. Every instance is
 * initialised exactly as lb_init would. Synchronises the stream. */
int lb_batch_init(lb_batch** b, const lb_batch_desc* d, int n, void* dev_workspace,
                  size_t workspace_bytes, void* stream);

/* Advance every instance by nsteps. By default one launch of the fused step
 * per step covers all instances (each block belongs to one instance); in
 * the persistent mode (lb_batch_set_persistent) one launch covers all
 * instances for 32 steps. Runs of 32 steps are replayed from a captured
 * CUDA graph on a private stream ordered after and before `stream`.
 * Asynchronous. Results per instance are identical to stepping the instance
 * alone with the same block size. */
int lb_batch_step(lb_batch* b, int nsteps);

/* Launch shape shared by all instances: block_x 64 or 128; seg_rows 0 gives
 * every instance a share of one full wave proportional to its cells. */
int lb_batch_set_launch(lb_batch* b, int block_x, int seg_rows);

/* Persistent mode (the batched boiling curve of Sec. 3.2-3.3 in one launch
 * per run of steps). tiles_per_block = 0 returns to one launch per step.
 * With tiles_per_block >= 1 (<= 64), lb_batch_step advances every instance
 * through runs of 32 steps, each run ONE cooperative launch of a fixed grid
 * (at most the blocks that fit on the GPU at once) replayed from a captured
 * CUDA graph, and the rest of the steps in one more launch. The instances
 * are cut into tiles (a block's two column strips x a segment of rows;
 * with seg_rows 0 the segments give about tiles_per_block tiles per block),
 * the tiles are dealt out to the blocks (longest first to the least loaded
 * block), and a tile starts a step once every tile of its instance has
 * finished the previous one. Results are bit-identical to stepping each
 * instance alone with the same block size. Each of those waits polls a
 * device counter at most wait_limit times (<= 0: the default, about 1-2
 * seconds); a wait that runs out ends its block and latches LB_E_TIMEOUT,
 * which lb_batch_sync and lb_batch_heat_flux report (the instances are then
 * only partly advanced and must be reset). */
int lb_batch_set_persistent(lb_batch* b, int tiles_per_block, long long wait_limit);

/* Per-instance heat-flux statistics into arrays of n entries (any may be
 * NULL); see lb_heat_flux. Synchronises; reports faults as lb_batch_sync. */
int lb_batch_heat_flux(lb_batch* b, double* q_inst, double* q_mean, double* q_std,
                       int64_t* nsamples, int reset);

/* Per-instance state copies and parameter changes (see the single-instance
 * calls of the same name). */
int lb_batch_get_state(lb_batch* b, int i, float* fpost, float* theta, int on_device);
int lb_batch_set_state(lb_batch* b, int i, const float* fpost, const float* theta, int on_device);
/* Macroscopic fields of instance i, as lb_fields (its outputs are [Ly_i*Lx_i]). */
int lb_batch_fields(lb_batch* b, int i, float* rho, float* ux, float* uy, float* T, int on_device);
int lb_batch_set_wall_temperature(lb_batch* b, int i, const double* Tb_profile, double superheat);
int lb_batch_set_wettability(lb_batch* b, int i, double Gw);

/* Steps taken, block size and blocks per launch (the persistent grid in
 * persistent mode). */
int lb_batch_info(lb_batch* b, int64_t* steps, int* block_x, int* nblocks);

/* Wait and report latched device faults of any instance: every instance's
 * flags are read and cleared, and the first fault found is returned. */
int lb_batch_sync(lb_batch* b);

/* Release the batch (the workspace stays the caller's). */
int lb_batch_destroy(lb_batch* b);

/* ---- pressure probes and the EOS pressure (Sec. 3.2, Fig. 3) ------------- */

/* Fig. 3 follows the pressure at the central point of the top wall while
 * bubbles rise and merge into the vapour above the pool. A probe records,
 * after every step t run through lb_step (and the forward pass of
 * lb_adjoint), the density rho^t, the temperature T^t = T_s + theta^t and
 * the pressure p = p_EOS(rho^t, T^t) of Eq. 21 at one cell: exactly the rho
 * and T the step used for psi there (rho^t is the sum of the stored
 * post-collision populations, which the collision conserves). With probes
 * set, each step is followed by one small single-block kernel.
 *
 * The ring is a caller-owned device buffer of lb_probe_ring_bytes(n,
 * capacity) bytes, 256-byte aligned: a 256-byte header, then for probe k
 * and record r the four floats (rho, T, p, 0) at float offset
 * 64 + 4 * (k * capacity + r). The s-th probed step (from 0, counted
 * since lb_set_probes) goes to record s % capacity, so the ring keeps the
 * last `capacity` steps; lb_probe_read returns them in time order. The
 * header's first 8 bytes are the count of probed steps (uint64). */
#define LB_PROBE_MAX 8

/* Ring bytes for n probes (1 <= n <= LB_PROBE_MAX) keeping `capacity`
 * steps (1 <= capacity <= 2^26): 256 + 16 n capacity. LB_E_INVAL outside. */
int lb_probe_ring_bytes(int n, int capacity, size_t* bytes);

/* Probe cells (x[k], y[k]), k < n <= LB_PROBE_MAX, 0 <= x < Lx, 0 <= y < Ly;
 * n = 0 removes the probes. Resets the ring's count. The ring must stay
 * allocated while probes are set. */
int lb_set_probes(lb_handle* h, int n, const int* x, const int* y, void* dev_ring, size_t ring_bytes,
                  int capacity);

/* Synchronises the handle's stream, then copies the newest m = min(count,
 * capacity, max_records) records of every probe, oldest first, into
 * out[k][j][0..2] = (rho, T, p) (host, n * m * 3 floats); *count = steps
 * probed since lb_set_probes, *m_out = m. Does not clear the ring. */
int lb_probe_read(lb_handle* h, int max_records, float* out, int64_t* count, int* m_out);

/* p_EOS(rho_i, T_i) of Eq. 21 for n host values, in FP64 (diagnostics:
 * pressure fields, the Laplace test of a bubble). */
int lb_eos_pressure(const lb_eos* eos, int64_t n, const float* rho, const float* T, double* p);

/* ---- no-allocation variant (not part of the paper's method) -------------- */

/* Largest grid (Lx * Ly cells) lb_fields_noalloc accepts. */
#define LB_NOALLOC_MAX_CELLS 262144

/* lb_fields without a handle, a workspace or any device allocation. The
 * paper has no counterpart; this exists for callers that cannot allocate
 * device memory themselves: code running inside another framework's memory
 * pool or allocator hook, processes that are not allowed to create
 * allocations after start-up, and real-time loops that must not touch the
 * allocator. Such a caller already holds the state in device memory and only
 * needs the macroscopic fields of it.
 *
 * Inputs (device pointers, unpitched, row-major as everywhere in this
 * header): fpost[9*Ly*Lx] post-collision populations and theta[Ly*Lx] =
 * T - T_s; rho_ave is the mean density at the start of the run (the
 * reference density of the buoyancy force) and Gw the strength of the
 * heating wall's fluid-solid force, both as given to lb_init. Outputs
 * (device, [Ly*Lx] each, any may be NULL): rho, ux, uy and T exactly as
 * lb_fields computes them. Grid fields other than Lx, Ly, bc_y and
 * ghost_layer, and the pool fields of th, are ignored.
 *
 * Scratch: the intermediate planes live in one static device array of
 * 4 * LB_NOALLOC_MAX_CELLS floats (4 MiB) plus 256 bytes inside the library.
 * Grids larger than LB_NOALLOC_MAX_CELLS are rejected with LB_E_INVAL. The
 * first call on a device looks up that array's device address (once per
 * device, with the device current); with the CUDA runtime's lazy module
 * loading (its default) that lookup also places the 4 MiB array in device
 * memory, so make the first call while that much device memory is still
 * free, and before starting any stream capture. Every GPU on which it has
 * been called keeps the array until the process exits. All calls share the
 * one array: calls that overlap on the GPU (other streams, other host
 * threads) race on it, so serialise them. The call is issued on `stream`
 * and synchronises it before returning; on a stream that is being captured
 * it enqueues nothing and returns LB_E_INVAL. It calls no cudaMalloc,
 * cudaFree or other allocating routine. Returns LB_E_EOS_DOMAIN if a cell's
 * density lies outside the domain of the equation of state. */
int lb_fields_noalloc(const lb_grid* grid, const lb_eos* eos, const lb_thermal* th,
                      double Gw, double rho_ave, const float* fpost, const float* theta,
                      float* rho, float* ux, float* uy, float* T, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* lb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LB_H */
