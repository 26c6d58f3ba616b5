/*
 * pic.h -- C-ABI of the GB300 (sm_103a) scattered-field particle-in-cell library.
 *
 * The library advances the scattered-field PIC cycle of Lytova et al. (arXiv
 * 2310.11393), Sec. 2 (the text after Eq. "scatt_field"): every macro-electron
 * gathers the grid-held scattered field (order-2 shapes, Sec. 3.1), adds the
 * closed-form incident field evaluated at its own position and time (plane wave
 * of Sec. 3.1; the tightly focused LP pulse of Sec. 4.1, Eqs. components,
 * phasor, poisson, poisson_dstr; the RP pulse generated by the Hertz vector
 * Psi z^ of the same Eq. phasor), takes a relativistic Boris push of the Lorentz
 * force in Eq. (vlasov), deposits an Esirkepov charge-conserving current, and
 * then the Yee scheme advances the scattered field only (Eqs. MAmper,
 * MFaraday).  Units are those of Table "tab:units": c = 1, omega = k = 1,
 * lengths in lambda/2pi, electron charge -1, mass 1, densities in n_c.
 *
 * Conventions common to every entry point
 *   - All calls return a pic_status; nothing aborts the process.  A failing call
 *     records a message readable with pic_last_error().
 *   - Pointers documented as HOST point to host memory owned by the caller and
 *     are not retained after the call returns.  DEVICE state is owned by the
 *     pic_sim and released by pic_destroy().
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls documented as asynchronous only enqueue work; errors found
 *     on the device (status word) surface at the next synchronous call.
 *   - Grid geometry: axis x (the propagation axis of every beam), then y, then z;
 *     `dim` resolved axes.  Node i of an axis sits at x = i*dx, i = 0..n; a field
 *     component staggered along an axis (Yee: E_c, J_c along c; B_c along the two
 *     other axes) has point i at (i + 1/2)*dx.
 *   - Field boundaries: first-order Mur absorbing faces.  Particles closer than
 *     `remove_margin` cells to a face leave the box (recorded as exits).
 *   - Thread safety: one pic_sim must not be used by two host threads at once.
 */
#ifndef SFFPIC_PIC_H
#define SFFPIC_PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = -1,      /* invalid argument or configuration */
    PIC_ENOMEM = -2,      /* device or host allocation failed */
    PIC_ECUDA = -3,       /* a CUDA runtime/driver call failed (message has the CUDA error) */
    PIC_ETIMEOUT = -4,    /* a bounded device wait gave up (status word bit PIC_FLAG_TIMEOUT) */
    PIC_ENAN = -5,        /* a non-finite value was found by a diagnostic */
    PIC_EBUSY = -6,       /* result not ready (serving) */
    PIC_ECAPACITY = -7,   /* a fixed-capacity buffer overflowed (exits, particles, admission) */
    PIC_ENODEV = -8,      /* no CUDA device of compute capability 10.3 available */
    PIC_ENOTFOUND = -9    /* unknown ticket / handle */
} pic_status;

/* PIC_BEAM_GAUSS2D: the 2D paraxial Gaussian beam of Sec. 3.2, Eq. (gauss2D) (dim 2 only):
 * waist w0, amplitude a0 = E0, FWHM_T = duration, envelope centre crossing the focus at
 * t_focus, carrier cos(Z - t + X^2/(2R) - eta + phi0); longitudinal field to first order in
 * 1/(k w0) including the wavefront-curvature term. */
enum { PIC_BEAM_NONE = 0, PIC_BEAM_PLANE = 1, PIC_BEAM_LP = 2, PIC_BEAM_RP = 3, PIC_BEAM_UNIFORM = 4,
       PIC_BEAM_GAUSS2D = 5 };
/* Slab density along x: uniform, or Sec. 3.1's super-Gaussian n0 2^-[2 (x - x0)/FWHM]^p beyond
 * a cut (0 before it); each electron's weight is n_e f(x)/ppc at its initial position. */
enum { PIC_PROFILE_UNIFORM = 0, PIC_PROFILE_SUPERGAUSS = 1 };
enum { PIC_ENV_SIN2 = 0, PIC_ENV_GAUSS = 1 };
/* PIC_FP64: every quantity in double precision.
 * PIC_FP32: particles, fields and the incident-field body in single precision; the
 * incident-field phase (t -/+ x against the focal point / reference plane) and
 * the particle coordinate it needs are formed in double precision first. */
enum { PIC_FP64 = 0, PIC_FP32 = 1 };

/* Momentum update: Boris (1970); Vay, Phys. Plasmas 15, 056701 (2008), which keeps the
 * force-free E x B drift of relativistic particles; Higuera & Cary, Phys. Plasmas 24,
 * 052104 (2017), which keeps it and is volume preserving. */
enum { PIC_PUSHER_BORIS = 0, PIC_PUSHER_VAY = 1, PIC_PUSHER_HC = 2 };

/* device status word bits (pic_info.status) */
enum {
    PIC_FLAG_TIMEOUT = 1u << 0,      /* an mbarrier wait exceeded its iteration bound */
    PIC_FLAG_CFL = 1u << 1,          /* a particle moved more than one cell in a step (removed) */
    PIC_FLAG_EXIT_OVERFLOW = 1u << 2, /* exit records beyond max_exits were dropped */
    PIC_FLAG_CAPACITY = 1u << 3       /* a particle found no slot in its destination tile and was
                                         dropped (the tile slack bounds the arrivals of a step,
                                         so this marks a defect, not a configuration limit) */
};

typedef struct {
    int32_t dim;             /* 1, 2 or 3 */
    int32_t n[3];            /* cells per axis (unused axes: 1) */
    double dx;               /* cell size, code units (lambda/2pi) */
    double dt;               /* time step; <= 0: cfl*dx/sqrt(dim) */
    double cfl;              /* used when dt <= 0; must keep dt < dx/sqrt(dim) */
    int32_t precision;       /* PIC_FP64 or PIC_FP32 */
    int32_t beam;            /* PIC_BEAM_* */
    int32_t envelope;        /* plane wave: PIC_ENV_SIN2 (sin^2 on [0, 2 FWHM]) or PIC_ENV_GAUSS (Sec. 3.1) */
    int32_t remove_margin;   /* cells; <= 0: 3 */
    double a0;               /* plane wave: field amplitude E0 = B0; LP/RP: peak of the on-axis focal
                                field envelope (LP: E_x, RP: E_z) used to derive Psi_0 */
    double duration;         /* field-amplitude FWHM (plane wave envelope; LP/RP on-axis focal envelope) */
    double w0;               /* LP/RP waist: k^2 w0^2 = 2(sqrt(1+(ka)^2)-1) gives a (Sec. 4.1) */
    double phi0;             /* constant phase (Eq. poisson) / plane-wave carrier phase */
    double t_focus;          /* LP/RP: time the pulse crosses the focus; Gaussian plane wave: centre */
    double focus[3];         /* LP/RP focus; plane wave: focus[0] is the plane where xi = t */
    double a_param;          /* LP/RP overrides, used when > 0 (else derived): a, s, Psi_0 */
    double s_param;
    double psi0;
    double e_unif[3];        /* PIC_BEAM_UNIFORM: constant external E and B */
    double b_unif[3];
    int32_t slab_lo[3];      /* electron slab, cells [lo, hi) per resolved axis */
    int32_t slab_hi[3];
    double n_e;              /* slab electron density (n_c) */
    int32_t ppc;             /* particles per slab cell (0: no slab) */
    int32_t tile[3];         /* particle tile in cells (2..248, x a multiple of 4); 0: chosen by the
                                autotuner */
    uint64_t seed;           /* SplitMix64 seed of the slab positions */
    int64_t max_particles;   /* particle capacity; 0: slab count (pic_set_particles may need more) */
    int64_t max_exits;       /* exit-record capacity; 0: max_particles */
    int32_t chunk;           /* particles per push work item (multiple of 256, 256..16384); 0: default */
    int32_t pusher;          /* PIC_PUSHER_*: momentum update of the Lorentz force (Sec. 2 cites all three) */
    int32_t profile;         /* PIC_PROFILE_*; the super-Gaussian uses prof_order (p >= 1), prof_x0,
                                prof_fwhm (> 0) and prof_cut, all in code units along x */
    int32_t prof_order;
    double prof_x0, prof_fwhm, prof_cut;
    int32_t tf_mode;         /* 1: total-field run (Sec. 3.1 case (i), 1D plane wave only): the
                                incident wave enters through the x = 0 face (its first-order
                                absorbing condition acts on E - E_inc) and is not added at the
                                particles; 0: scattered-field run */
    int32_t incident_grid;   /* 1: the incident field is evaluated once per step on the Yee nodes of
                                each component (the prescribed-field route of Smilei, Sec. 2 last
                                paragraph) and gathered with the scattered field, instead of at
                                every particle: 2^dim closed-form evaluations per cell instead of
                                ppc; interpolation error O((k dx)^2); 0: at the particle (Sec. 2) */
    int32_t autotune_steps;  /* > 0: pic_init first runs pic_autotune with this many trial steps
                                for a tile or chunk left at 0 (cached per shape) */
    int32_t sort_every;      /* cell sort within the tiles (a layout choice, no counterpart in the
                                paper): > 0: every sort_every-th step the tile re-sort also
                                orders each tile's particles by cell (x fastest), so that a
                                warp's lanes sit on neighbouring cells again; <= 0: never (the
                                push measured no faster on sorted tiles).  Costs two arrays of
                                one int per cell of the tiled grid.  Changes only the order of
                                the particles (and with it the rounding order of the deposit). */
} pic_config;

/* Host-side derived quantities (pic_derive_params, pic_info). */
typedef struct {
    double a, s, psi0;       /* LP/RP pulse parameters (0 for other beams) */
    double dt;               /* time step actually used */
    int64_t n_particles;     /* seeded slab particles */
    int64_t device_bytes;    /* device memory pic_init will request */
    int32_t tile[3];         /* particle tile after autotuning */
    int32_t yee_tile[3];     /* field-solver tile (3D: x, y of a column and its segment in z) */
    int32_t chunk;           /* particles per push work item */
    int32_t sort_every;      /* steps between cell sorts (0: none) */
} pic_params;

typedef struct {
    int64_t step;            /* steps taken */
    double time;             /* step * dt */
    int64_t n_alive;         /* particles in the box */
    int64_t n_exits;         /* exit records stored */
    uint32_t status;         /* PIC_FLAG_* bits seen so far */
    pic_params params;
} pic_info;

/* Device memory provider.  alloc(bytes, ctx) returns device memory (256-byte aligned)
 * or NULL; free(ptr, ctx) releases it.  Both are called only on the calling thread, from
 * pic_init and pic_destroy, and from pic_batch_step for the launch tables of a new list of
 * simulations (taken from its first member's provider and given back when any member is
 * destroyed).  A NULL pic_allocator* means cudaMalloc/cudaFree. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
} pic_allocator;

typedef struct pic_sim pic_sim;

/* ---- parameters (host only, no device needed) ------------------------------------ */
/* Validates cfg and fills out: a from w0 (Sec. 4.1 waist relation), s from `duration`
 * (field FWHM of the on-axis focal envelope), Psi_0 from a0 (peak of that envelope),
 * dt, particle count, tiles and the device footprint.  Returns PIC_EINVAL with a
 * message for an invalid configuration. */
pic_status pic_derive_params(const pic_config* cfg, pic_params* out);

/* ---- lifecycle ------------------------------------------------------------------- */
/* Creates a simulation on the current CUDA device: allocates its device state through
 * `alloc`, places the seeded slab (SplitMix64, particle p uses outputs 3p+d; offset =
 * top 24 bits / 2^24), zeroes the scattered field and captures the step as a CUDA
 * graph.  Synchronous on `stream`.  *out is NULL on failure. */
pic_status pic_init(const pic_config* cfg, const pic_allocator* alloc, void* stream, pic_sim** out);

/* Autotuner of the particle tile and the push work-item size (no counterpart in the paper:
 * a layout choice of this implementation).  For each candidate (tiles of 8..32 cells per
 * axis by dimension, then work items of 256..4096 particles at the best tile) it creates
 * the simulation on the current device and times two stretches, each trial_steps untimed
 * steps and then the faster of two runs of trial_steps timed steps (CUDA events on
 * `stream`): one from t = 0, one around the time the pulse is on the plasma (focused beams:
 * at the focus; plane wave: envelope centre at the slab centre), reached by stepping when
 * that takes at most 1500 steps (electrons heated by the pulse, as in the run) and else by
 * moving the clock, so that the incident field and the deposit do their full work; the
 * candidate's time is the mean of the two.  It then destroys it; one
 * candidate holds device memory at a time.  The tiles are timed at work items of 4096 for a
 * run of at least 16 such work items per SM and of 2048 otherwise; a later candidate must be
 * faster by more than 1 % to be chosen.  Candidates that do not fit (shared memory,
 * device memory) are skipped.  On success cfg->tile and cfg->chunk hold the fastest
 * choice and *ms_per_step (may be NULL) its time per step.  Only tile/chunk entries left
 * at 0 are tuned.  Results are cached for the process per (dim, precision, n, ppc, beam,
 * slab): a repeated call returns the cached choice without measuring.
 * Errors: PIC_EINVAL (bad config, trial_steps < 1), PIC_ENODEV, or the first candidate's
 * pic_init error when no candidate could be created. */
pic_status pic_autotune(pic_config* cfg, int trial_steps, void* stream, double* ms_per_step);

/* Advances n_steps >= 0 steps (one step: push + current deposition with every particle
 * placed straight into its destination tile of the other particle buffer set, tile scan,
 * field update).  Asynchronous on `stream` (graph replays).  Every sort_every-th step
 * taken through pic_step or pic_profile_step (counted per sim from pic_init) replays the
 * variant that places each tile's particles in cell order. */
pic_status pic_step(pic_sim* sim, int n_steps, void* stream);

/* Advances n_steps steps like pic_step but launches the kernels one by one with CUDA
 * events recorded on `stream` between the phases, and returns in HOST seconds[5] the
 * summed device time of each phase: [0] push + deposit (with incident_grid: also the
 * evaluation of the incident field on the grid), [1] tile scan, [2] cell-sort placement
 * (zero on other steps), [3] field solve, [4] step end (with the next step's chunk
 * numbering).  Synchronous.  Used to time kernels live. */
pic_status pic_profile_step(pic_sim* sim, int n_steps, void* stream, double* seconds);

/* Releases all device state; synchronises the simulation's work first.  NULL is a no-op. */
pic_status pic_destroy(pic_sim* sim);

/* Message of the last failing call on `sim` (or of the calling thread when sim is NULL).
 * The string stays valid until the next call on the same sim / thread. */
const char* pic_last_error(const pic_sim* sim);

/* Step counter, particle counts and status word.  Synchronises `stream`. */
pic_status pic_info_get(pic_sim* sim, pic_info* out, void* stream);

/* ---- explicit state (inputs, checkpoint / restore) -------------------------------- */
/* Replaces every particle.  HOST arrays: x[n][3] grid coordinates (unused axes ignored),
 * u[n][3] momenta (gamma v), w[n] weights (density per particle, n_c), id[n] >= 0 and
 * < 2^31.  Particles must lie inside the box, at least remove_margin cells from every
 * face (else PIC_EINVAL).  n may exceed the slab count up to max_particles.
 * Synchronous on `stream`. */
pic_status pic_set_particles(pic_sim* sim, int64_t n, const double* x, const double* u,
                             const double* w, const int64_t* id, void* stream);

/* Replaces the grid fields.  HOST array of 9 components (Ex Ey Ez Bx By Bz Jx Jy Jz),
 * each ext_z*ext_y*ext_x doubles, x fastest, ext = n+1 on resolved axes and 1 otherwise;
 * points a component does not have (index n along a staggered axis) are ignored.
 * The magnetic field is the one at the same integer time as E.  Synchronous. */
pic_status pic_set_fields(pic_sim* sim, const double* fields, void* stream);

/* Moves the step counter (time = step * dt); used with restored state.  Synchronous. */
pic_status pic_set_step(pic_sim* sim, int64_t step, void* stream);

/* ---- diagnostics (synchronous on `stream`; HOST output owned by the caller) -------- */
enum {
    PIC_DIAG_ENERGIES = 0,   /* double[8]: EM energy of the scattered field, EM energy of scattered +
                                incident field on the grid points, kinetic energy sum w(gamma-1)dx^dim
                                of the electrons in the box, kinetic energy carried out by exits,
                                n_alive, n_exits, step, time */
    PIC_DIAG_GAUSS = 1,      /* double[1]: max |div E - rho_e - rho_ion| over interior nodes, with
                                rho_ion = -rho_e at step 0 (immobile ions) */
    PIC_DIAG_PARTICLES = 2,  /* n_alive records of 8 doubles: x[3], u[3], w, id (as double) */
    PIC_DIAG_EXITS = 3,      /* n_exits records of 6 doubles: u[3] at exit, w, id, step of exit */
    PIC_DIAG_FIELDS = 4      /* double[9][ext_z][ext_y][ext_x] as in pic_set_fields (absent points 0) */
};
/* Writes diagnostic `kind` into host_out, which must hold at least the bytes the kind
 * needs (PIC_ECAPACITY otherwise; pic_info_get gives the counts).  Returns PIC_ETIMEOUT
 * if the device status word has the timeout bit, PIC_ECAPACITY if it has the capacity
 * bit, PIC_ENAN if an energy is not finite. */
pic_status pic_diag(pic_sim* sim, int kind, void* host_out, size_t bytes, void* stream);

/* Weighted electron histogram over kinetic energy gamma-1 in [0, e_max) (n_e bins) and
 * angle from the +x (propagation) axis in [0, pi] (n_a bins); electrons in the box plus
 * exits.  HOST output: double[n_e * n_a], angle fastest.  Runs on the simulation's device
 * (made current for the call).  Synchronous.  Returns PIC_ETIMEOUT / PIC_ECAPACITY for the
 * device status word's timeout / capacity bits, as pic_diag. */
pic_status pic_histogram(pic_sim* sim, int n_e, double e_max, int n_a, double* host_out, void* stream);

/* Same weighted energy-angle histogram as pic_histogram, for callers that must not allocate
 * device memory on the call path: for example a serving loop whose device memory is fully
 * claimed by a framework's caching allocator, or a real-time loop that must not risk the
 * device-wide synchronisation that cudaMalloc / cudaFree can cause.  It allocates nothing: the
 * bins are accumulated in a file-scope device array of PIC_HIST_STATIC_MAX_BINS doubles
 * (128 KiB) that every GPU which loads the library holds until the process exits.  The first
 * call on a device looks the array up (cudaGetSymbolAddress) with that device current, so make
 * that first call before any stream capture.  Every call clears the bins it uses and then
 * leaves its result in the array; calls that overlap on the GPU (different streams or host
 * threads) share the array and race, so serialise them.  n_e * n_a > PIC_HIST_STATIC_MAX_BINS
 * is rejected with PIC_EINVAL.  HOST output double[n_e * n_a], angle fastest.  Runs on the
 * simulation's device (made current for the call, including the first call's look-up); the
 * status word is read as pic_diag reads it (PIC_ETIMEOUT, PIC_ECAPACITY).  Synchronous.
 * (No counterpart in the paper: this is an interface for constrained callers.) */
#define PIC_HIST_STATIC_MAX_BINS 16384
pic_status pic_histogram_static(pic_sim* sim, int n_e, double e_max, int n_a, double* host_out, void* stream);

/* Evaluates the simulation's incident field with the device code path at n HOST points
 * pts[n][4] = (x, y, z, t) in grid coordinates; HOST out[n][6] = Ex Ey Ez Bx By Bz.
 * Synchronous.  Used to check the incident-field arithmetic point by point. */
pic_status pic_eval_incident(pic_sim* sim, int64_t n, const double* pts, double* out, void* stream);

/* ---- batching: many independent simulations per launch --------------------------- */
/* Advances every sim by n_steps: one persistent launch per phase over all their tiles
 * (sims grouped by dim and precision), the whole step captured as one CUDA graph that is
 * cached for this exact list.  All sims must live on the current device.  Asynchronous.
 * The cell sort runs for every member that has one every k-th call step of this list,
 * k the smallest sort_every among the members (counted per cached list). */
pic_status pic_batch_step(pic_sim** sims, int n_sims, int n_steps, void* stream);

/* Advances the same list n_steps steps like pic_batch_step, but launches each phase of the
 * step (over every launch group of the list) one after another, with CUDA events recorded on
 * `stream` between the phases, and returns in HOST seconds[5] the summed device time of each
 * phase, as pic_profile_step.  Synchronous.  Used to compare the batched path with the plain
 * one phase by phase. */
pic_status pic_batch_profile_step(pic_sim** sims, int n_sims, int n_steps, void* stream, double* seconds);

/* ---- serving: continuous batching of a request stream ----------------------------- */
typedef struct pic_server pic_server;
typedef struct {
    int64_t memory_budget;   /* device bytes the resident simulations may use; 0: 80% of free memory */
    int32_t max_resident;    /* simulations on the device at once; 0: 256 */
    int32_t quantum;         /* steps advanced between admission rounds; 0: 50 */
    int64_t fill_particles;  /* each quantum steps the resident simulations with the least
                                remaining work (steps x electrons) first, adding more until
                                this many electrons are in the batch (enough to fill the GPU);
                                the others wait for the next quantum.  A batch of one steps
                                through that simulation's own step graph.  0: 2 000 000;
                                < 0: all */
} pic_serve_config;
typedef struct {
    int32_t state;           /* 0 queued, 1 running, 2 done, -1 failed */
    int32_t error;           /* pic_status of a failed request */
    int64_t steps_done;
    double submit_time;      /* seconds on the server clock */
    double start_time;
    double finish_time;
    double energies[8];      /* PIC_DIAG_ENERGIES at completion */
    int64_t pushes;          /* particle pushes performed */
} pic_result;

/* Starts a server with a host scheduling thread on the current device. */
pic_status pic_serve_open(const pic_serve_config* cfg, pic_server** out);
/* Queues a simulation request of n_steps; *ticket identifies it.  Thread safe. */
pic_status pic_serve_submit(pic_server* srv, const pic_config* cfg, int64_t n_steps, uint64_t* ticket);
/* Fills *out; returns PIC_EBUSY while the request is queued or running. Thread safe. */
pic_status pic_serve_poll(pic_server* srv, uint64_t ticket, pic_result* out);
/* Seconds on the server clock (the clock of pic_result times). */
double pic_serve_clock(const pic_server* srv);
/* Finishes running requests, stops the thread, frees everything. */
pic_status pic_serve_close(pic_server* srv);

/* ---- test aid (no counterpart in the paper) --------------------------------------- */
/* Fault injection for the bounded device waits, without faulting the GPU: block `block` of
 * the single-simulation tile scan (which scans 4096 particle tiles per block and chains the
 * blocks by decoupled look-back) stops publishing its totals, so the blocks after it poll
 * its flag `spins` times (default 2^22, about a second), give up, set PIC_FLAG_TIMEOUT in
 * the status word and take a zero prefix, which keeps every later offset inside the
 * particle arrays (the particle layout is then wrong, and the next synchronous call returns
 * PIC_ETIMEOUT).  block = -1 restores publishing.  Only simulations with more than 4096
 * particle tiles use the multi-block scan.  Synchronous.  Errors: PIC_EINVAL (spins < 1),
 * PIC_ECUDA. */
pic_status pic_test_hold_scan(pic_sim* sim, int block, int spins);

/* ---- measurement aid (no counterpart in the paper) -------------------------------- */
/* Issue rates of the current device measured with CUDA events over all SMs: dependency
 * chains of FP32 fused multiply-adds (8 independent chains per thread, the loop unrolled
 * 16 times), of FP64 fused multiply-adds and of the special-function unit's approximate
 * sine.  fp32_tflops counts an FMA as two operations; sfu_gops counts one per sine.  The SM
 * clock is clock64() cycles of the longest block over the event time of the FP32 probe,
 * and fp32_flop_per_clk_sm the FP32 rate per SM and clock it implies.  The fused push's
 * transcendental-heavy closed form is bound by these rates rather than by HBM, so they
 * are its roofline.  About 0.2 s of GPU time; allocates 64 bytes plus 8 per block with
 * cudaMalloc.  Synchronous on `stream`.  Errors: PIC_ENODEV, PIC_ENOMEM, PIC_ECUDA. */
typedef struct {
    int32_t sms;             /* streaming multiprocessors of the device */
    double fp32_tflops;
    double fp64_tflops;
    double sfu_gops;
    double sm_clock_mhz;
    double fp32_flop_per_clk_sm;
} pic_peaks;
pic_status pic_probe_peaks(pic_peaks* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFFPIC_PIC_H */
