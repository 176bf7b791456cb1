/*
 * pic.h -- C ABI of libpic: the 3D particle-in-cell time step on a Yee FDTD
 * grid with Drude metals, after "Numerical study of three-dimensional PIC for
 * the surface plasmon excitation based on Drude model" (Liu, Zhao, Wang, Liu).
 *
 * One time step n -> n+1 (Sec. II; the particle-field coupling is the usual
 * Yee PIC one, Sec. II last paragraph):
 *   1. H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n                    (vacuum Yee)
 *      with convolutional-PML (CPML) terms in the absorbing face slabs;
 *   2. electrons: staggered trilinear gather of E^n and
 *      B^n = mu0 (H^{n-1/2} + H^{n+1/2})/2, relativistic Boris push,
 *      x^{n+1} = x^n + dt u/gamma (u = gamma v);
 *   3. charge-conserving (Esirkepov) free current J_f^{n+1/2};
 *   4. Drude polarisation current, Eq. 6 (E read at level n):
 *        J^{n+1/2} = (2-g dt)/(2+g dt) J^{n-1/2} + 2 dt eps0 wp^2/(2+g dt) E^n
 *      then Eq. 8: E^{n+1} = E^n + dt/(eps0 eps_inf)[curl H^{n+1/2} - J^{n+1/2} - J_f^{n+1/2}];
 *   5. probe DFT: F[p][c][f] += E_c^{n+1}(x_p) exp(+i 2 pi f (n+1) dt) dt.
 *
 * Conventions for every call:
 *  - SI units.  Arrays of the grid are [nz][ny][nx] with x fastest.
 *  - Yee staggering: Ex (i+1/2,j,k)  Ey (i,j+1/2,k)  Ez (i,j,k+1/2)
 *                    Hx (i,j+1/2,k+1/2)  Hy (i+1/2,j,k+1/2)  Hz (i+1/2,j+1/2,k)
 *    On a non-periodic axis the outer faces are node 0 and node n; tangential
 *    E on them is held at zero.
 *  - Every call returns PIC_OK (0) or a negative PIC_ERR_* code; the message
 *    of the last failure on the calling thread is pic_last_error().
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Output host arrays are written before return.
 *  - Device work runs on the handle's stream (pic_config.stream or
 *    pic_set_stream).  pic_step is asynchronous; calls that return data to the
 *    host synchronise that stream and report device-side errors.
 *  - A handle is not thread-safe: one thread at a time per handle.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_ERR_ARG -1         /* invalid argument or out-of-range input */
#define PIC_ERR_CFL -2         /* dt violates the Yee + Drude stability bound */
#define PIC_ERR_OOM -3         /* device allocation or workspace too small */
#define PIC_ERR_CUDA -4        /* a CUDA runtime call failed */
#define PIC_ERR_NONFINITE -5   /* a NaN/Inf was detected in the state */
#define PIC_ERR_STATE -6       /* call not valid in the handle's current state */
#define PIC_ERR_UNSUPPORTED -7 /* configuration outside what the library implements */
#define PIC_ERR_DEVICE -8      /* a kernel reported an internal error */

enum { PIC_FP32 = 0, PIC_FP64 = 1 };
enum { PIC_BC_CPML = 0, PIC_BC_PEC = 1, PIC_BC_PERIODIC = 2 };
enum {
    PIC_EX = 0, PIC_EY, PIC_EZ,
    PIC_HX, PIC_HY, PIC_HZ,
    PIC_JPX, PIC_JPY, PIC_JPZ, /* Drude polarisation current (Eq. 6) */
    PIC_JFX, PIC_JFY, PIC_JFZ  /* free (particle + source) current of the last step */
};

/* Drude parameters of one material id (Eq. 1): plasma frequency wp [rad/s],
 * collision rate gamma [1/s], high-frequency permittivity eps_inf (1 in the
 * paper).  wp = 0 is a plain dielectric (vacuum when eps_inf = 1). */
typedef struct {
    double wp;
    double gamma;
    double eps_inf;
} pic_material;

typedef struct {
    int64_t nx, ny, nz;           /* cells per axis, each >= 1 */
    double dx, dy, dz;            /* cell size [m] */
    double dt;                    /* time step [s] */
    double eps0, mu0;             /* vacuum constants [F/m], [H/m] */
    int32_t precision;            /* PIC_FP32 (fields, J, particles in float) or PIC_FP64 */
    int32_t bc[6];                /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi: PIC_BC_*; periodic must pair */
    int32_t cpml_cells;           /* absorbing slab thickness L in cells */
    double cpml_order;            /* grading exponent m */
    double cpml_sigma_fac;        /* sigma_max = fac (m+1)/(eta0 d) */
    double cpml_kappa_max;        /* kappa at the outer face (1 = no stretching) */
    double cpml_alpha_max;        /* CFS shift at the inner face [S/m] */
    const uint8_t *material_id;   /* host [nz][ny][nx] ids into materials[] */
    const pic_material *materials;
    int32_t n_materials;          /* 1..256 */
    int64_t max_particles;        /* capacity reserved at create */
    int32_t max_probes;           /* capacity for pic_probe_dft */
    int32_t max_freqs;
    void *workspace;              /* optional caller-owned device memory (NULL: library allocates) */
    size_t workspace_bytes;       /* size of workspace, >= pic_workspace_size() */
    void *stream;                 /* cudaStream_t for all device work (NULL: a stream the library creates) */
    uint64_t flags;               /* PIC_FLAG_* bits, else 0 */
} pic_config;

/* pic_config.flags: keep the FP32 field updates as two separate passes (the
 * H update, then the E update) on a grid that would take the fused pass.
 * The fused pass: FP32 grids with nx a multiple of 4, no periodic axis and,
 * where an axis has absorbing layers, cpml_cells <= 8 (a multiple of 4 along
 * x) and more than 32 + cpml_cells cells along x, 15 + cpml_cells along y,
 * advance E (Eq. 6 then Eq. 8) and the next step's H in one sweep over the
 * grid (48 instead of 72 bytes per cell), holding two copies of the field
 * state (the arena is larger by one copy of E, H, J, J_f and the CPML
 * memory); the results are those of the split updates up to rounding order. */
#define PIC_FLAG_SPLIT_FIELDS 1

/* pic_config.flags: copy the caller's host arrays (the material map here,
 * positions and momenta in pic_add_particles) through the CUDA runtime.
 * Without it, on a device that reads pageable host memory coherently
 * (cudaDevAttrPageableMemoryAccess, e.g. a Grace system) kernels read them
 * where they are, before the call returns; elsewhere they are copied either
 * way.  The results are the same. */
#define PIC_FLAG_STAGED_UPLOAD 2

typedef struct {
    int64_t step;          /* completed time steps */
    int64_t n_particles;   /* particles added */
    int64_t n_frozen;      /* particles stopped by the boundary/metal rule */
    int32_t device_error;  /* bits (0 = none): 1 an electron moved more than one cell in
                              a step (impossible under the time-step bound pic_create
                              checks: a guard against a corrupted state); 2 an electron's
                              momentum became non-finite (it is frozen); 4 E or H holds
                              a NaN or an Inf (found by the scan of pic_sync and
                              pic_get_stats); 8 a wait of the fused field pass for its
                              staged planes ran out of time (the pass stopped early).
                              Bits stay set for the life of the handle. */
    int32_t n_edge_classes;
    int64_t kernel_launches; /* kernels pic_step has launched (graph replays count their kernels) */
    int32_t field_path;    /* 1: the fused FP32 field pass (see PIC_FLAG_SPLIT_FIELDS); 0: split updates */
    int32_t reserved;
} pic_stats;

typedef struct pic_handle pic_handle;

/* Message for the last failing call on this thread ("" if none).  The
 * string stays valid until the thread's next library call. */
const char *pic_last_error(void);

/* Device bytes pic_create needs for cfg (grid state, particles and probe
 * capacity).  Nothing is allocated.  Errors: PIC_ERR_ARG on an invalid cfg. */
int pic_workspace_size(const pic_config *cfg, size_t *bytes);

/* Build a simulation: validates sizes and the stability bound
 * c^2 dt^2 sum(1/d^2) + wp_max^2 dt^2/4 < 1, derives the per-edge Drude
 * coefficients of Eq. 6 and the Ampere factor of Eq. 8 from the material map
 * (wp^2 on an edge is the mean over the four cells sharing it, gamma its
 * wp^2-weighted mean, eps_inf the plain mean), builds the CPML profiles, and
 * zeroes E, H, J.  Device memory comes from cfg->workspace if given (the
 * caller keeps it alive until pic_destroy), else from cudaMalloc.
 * *out receives an opaque handle owned by the library until pic_destroy.
 * Errors: PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_OOM, PIC_ERR_UNSUPPORTED (more
 * than 256 distinct edge materials, 2^32 cells or more, ny above 262140 or
 * nz above 131070), PIC_ERR_CUDA. */
int pic_create(const pic_config *cfg, pic_handle **out);

/* Release the handle and any memory the library allocated.  Waits for the
 * handle's stream.  NULL is accepted. */
int pic_destroy(pic_handle *h);

/* Use another cudaStream_t for subsequent device work (NULL: a stream the
 * library creates and owns).  Waits for the old stream; drops captured step
 * graphs.  The legacy default stream cannot be captured into graphs, so pass
 * a created stream, not 0, when sharing one. */
int pic_set_stream(pic_handle *h, void *stream);

/* Append n macro-electrons of the bunch (Sec. III: an electron bunch moving
 * parallel to the film surface excites its surface plasmons; the electrons
 * then take part in every step as in Sec. II's particle-field coupling):
 * xyz [n][3] positions [m], u [n][3] gamma*v [m/s],
 * charge q_macro [C] (negative for electrons) and mass m_macro [kg] of each
 * (all particles of a handle share q and m).  Every position must lie at
 * least two cells inside each non-periodic face and outside cells with
 * wp > 0; otherwise nothing is added, *n_rejected (if non-NULL) receives the
 * count of particles breaking the first of these two rules that some particle
 * breaks, and PIC_ERR_ARG is returned.  Positions on
 * periodic axes are wrapped.  Exceeding max_particles is PIC_ERR_OOM. */
int pic_add_particles(pic_handle *h, int64_t n, const double *xyz, const double *u,
                      double q_macro, double m_macro, int64_t *n_rejected);

/* Read particles back in the order they were added: xyz [n][3] (m),
 * u [n][3] (m/s), status [n] (0 live, 1 frozen).  Any pointer may be NULL.
 * Synchronises. */
int pic_get_particles(pic_handle *h, double *xyz, double *u, uint8_t *status);

/* 1: electrons deposit current (default).  0: they are test particles that
 * feel the fields but do not drive them. */
int pic_set_deposit(pic_handle *h, int on);

/* Prescribed current density added to J_f on the edges of component comp
 * (0..2) with indices box = {i0,i1,j0,j1,k0,k1} (half-open) at every step:
 * amp * exp(-s^2) * sin(2 pi f0 (t-t0)) for f0 > 0, amp * (-2 s) exp(-s^2)
 * for f0 == 0, s = (t-t0)/tau, evaluated at t = (n+1/2) dt.  At most 16. */
int pic_add_source(pic_handle *h, int comp, const int64_t *box, double amp, double t0,
                   double tau, double f0);

/* Configure the probe DFT (Sec. IV, the spectrum of the field above the
 * film): np points xyz [np][3] (m), components comp_mask (bit c = E_c),
 * nf frequencies freq_hz [nf].  Zeroes the accumulators.  Points must lie at
 * least one cell inside each non-periodic face.  Capacity: max_probes,
 * max_freqs. */
int pic_probe_dft(pic_handle *h, int np, const double *xyz, uint32_t comp_mask, int nf,
                  const double *freq_hz);

/* Advance nsteps time steps of the method of Sec. II: per step the vacuum Yee
 * H update, the electron push and charge-conserving current, then the Drude
 * current of Eq. 6 before the E update of Eq. 8 (J first, then E, as the
 * paper orders them), then the probe sample (the five stages listed at the top
 * of this file).  Asynchronous on the handle's stream; device-side errors
 * are reported by the next synchronising call.  Steps are grouped into
 * blocks of 64 (one probe-DFT flush each): whole blocks replay one captured
 * CUDA graph; a run of 8..63 steps inside a block launches kernel by kernel
 * the first time it is asked for and replays a graph captured the second
 * time (runs are told apart by where in the block they start; the 16 most
 * recently used are kept per handle); shorter runs launch kernel by kernel.  The arithmetic is the same on every
 * route.  Errors: PIC_ERR_ARG (nsteps < 0), PIC_ERR_CUDA (launch or capture
 * failed). */
int pic_step(pic_handle *h, int64_t nsteps);

/* Wait for the handle's stream, then scan E and H for NaN or Inf (one pass
 * over the six arrays).  Returns PIC_ERR_DEVICE if a kernel set error bit 1,
 * 2 or 8 (see pic_stats.device_error), else PIC_ERR_NONFINITE if E or H holds
 * a non-finite value, else PIC_OK. */
int pic_sync(pic_handle *h);

/* Copy the probe spectra to out [np][3][nf][2] (re, im; components not in
 * the mask are zero).  Synchronises. */
int pic_probe_read(pic_handle *h, double *out);

/* Space-time spectrum of the probe line (the paper's dispersion picture,
 * Sec. II / Fig. 2): for the wavenumbers k[0..nk) (rad/m) along axis `axis`
 * (0 x, 1 y, 2 z),
 *     out[q][f] = | sum_p F[p][comp][f] exp(-i k[q] s_p) |^2   (nk x nf, row-major)
 * with F the probe spectra of pic_probe_read and s_p the coordinate of probe
 * p along the axis in metres.  Meaningful for probes on a line along that
 * axis.  Flushes buffered samples; synchronises; allocates two temporary
 * device buffers (k and out).  Errors: PIC_ERR_STATE (no probes), PIC_ERR_ARG
 * (comp/axis out of range, nk > 65535, NULL arrays), PIC_ERR_OOM, PIC_ERR_CUDA. */
int pic_probe_kw(pic_handle *h, int comp, int axis, int nk, const double *k, double *out);

/* Copy grid array `which` (PIC_EX..PIC_JFZ) to out [nz][ny][nx] as double.
 * Synchronises. */
int pic_get_field(pic_handle *h, int which, double *out);

/* Overwrite E or H component `which` (PIC_EX..PIC_HZ) from in [nz][ny][nx]
 * (rounded to the state precision).  Used for initial conditions and
 * restarts.  Synchronises. */
int pic_set_field(pic_handle *h, int which, const double *in);

/* Counters and the device error word (after the same scan of E and H as
 * pic_sync).  Synchronises. */
int pic_get_stats(pic_handle *h, pic_stats *out);

/* Write the complete state of the simulation to the file `path`: fields,
 * J, CPML memory, particles, probe accumulators and buffered samples, sources
 * and the step counter (the whole device arena plus the host-side counters).
 * Synchronises.  Errors: PIC_ERR_ARG (file cannot be written), PIC_ERR_CUDA. */
int pic_save(pic_handle *h, const char *path);

/* Restore a state written by pic_save into h, which must have been created
 * with the same configuration (grid, precision, boundaries, materials,
 * capacities); stepping then continues exactly where the saved run stood
 * (up to the summation order of atomic current deposits).  Synchronises.
 * Errors: PIC_ERR_ARG (missing/truncated file or a different configuration),
 * PIC_ERR_CUDA. */
int pic_load(pic_handle *h, const char *path);

/* Time the given number of steps with CUDA events placed between the phases
 * of steps run exactly as pic_step runs them (the push and deposit overlap
 * the E update on a second stream, the absorbing-slab part of each field
 * update runs beside the interior part).  Returns per-step averages in
 * microseconds: out[0] H update (from the start of the step to the end of
 * the H update on both streams), out[1] push + deposit (its own stream),
 * out[2] E update (both streams), out[3] wait for the deposit + free-current
 * term + probe sampling, out[4] probe DFT flush per step, out[5] whole step
 * (without the brick sort that precedes every 16th step).  On the fused
 * path (pic_stats.field_path 1) the phases are: out[0] the fused field pass
 * (E and the next step's H, all four tile kinds), out[1] push + deposit +
 * sources (before the pass), out[2] the free-current correction, out[3]
 * probe sampling, out[4] and out[5] as above.  Runs real steps (the simulation advances).
 * Synchronises. */
int pic_profile_steps(pic_handle *h, int64_t nsteps, double *out_us);

/* ---------------------------------------------------------------- tuning --
 * Launch settings that change how fast a step runs, never what it computes
 * (the paper has no counterpart; results stay those of pic_step up to the
 * summation order of the atomic current deposits):
 *   dep_smem_bytes  largest node box (three current components) a block of
 *                   the deposit accumulates in shared memory before adding
 *                   it to J_f; blocks whose electrons span more nodes add
 *                   straight to J_f.  0 .. 16384, a multiple of 16.
 *                   Default 4096.
 *   sort_every      electrons are re-sorted by 4x4x4-cell brick every this
 *                   many steps: 1, 2, 4, 8, 16, 32 or 64.  Default 16.
 *   field_block     threads per block of the FP32 field kernels of the cells
 *                   away from the absorbing slabs (the H update, and the E
 *                   update on planes without metal; four x cells per thread,
 *                   blocks taken in turn over the boxes of the grid): 128, 256
 *                   or 512.  Default 256.  No effect on the FP64 state or on
 *                   grids the four-cell kernels do not take.
 *   field_path      1: the fused field pass (see PIC_FLAG_SPLIT_FIELDS) on a
 *                   grid that takes it; 0: the H and E updates as two
 *                   passes.  Default 1.  A handle whose grid does not take
 *                   the fused pass (or created with PIC_FLAG_SPLIT_FIELDS)
 *                   accepts 1 and reports 0.
 * The settings belong to the handle, not to the simulation state: pic_save
 * does not write them and pic_load leaves the handle's settings as they are. */
typedef struct {
    int32_t dep_smem_bytes;
    int32_t sort_every;
    int32_t field_block;
    int32_t field_path;
} pic_tuning;

/* The handle's current launch settings into *out.  Errors: PIC_ERR_ARG (NULL). */
int pic_get_tuning(pic_handle *h, pic_tuning *out);

/* Errors: PIC_ERR_ARG (NULL or a value outside the ranges above). */
int pic_set_tuning(pic_handle *h, const pic_tuning *t);

/* Candidates pic_tune times: dep_smem_bytes over {0, 2048, 4096, 8192, 16384}
 * with the rest held, then sort_every over {8, 16, 32, 64} with the best box,
 * then field_block over {128, 256, 512} with the best box and interval, then
 * (on a grid that takes the fused pass) field_path {1, 0}. */
#define PIC_TUNE_MAX_CANDIDATES 20
typedef struct {
    pic_tuning best;
    int32_t n;                                    /* candidates timed */
    pic_tuning cand[PIC_TUNE_MAX_CANDIDATES];
    double us_per_step[PIC_TUNE_MAX_CANDIDATES];  /* best block of each, per step */
    int64_t steps;                                /* simulation steps taken */
    int32_t best_lanes;                           /* pic_batch_tune: chosen lanes (else -1) */
    int32_t lanes[PIC_TUNE_MAX_CANDIDATES];       /* pic_batch_tune: lanes of each candidate (else -1) */
} pic_tune_report;

/* Choose the tuning for this simulation by timing it: `rounds` (1..16)
 * passes of the candidates above, each candidate stepping one whole 64-step
 * block (CUDA events on the simulation's stream); each candidate keeps its
 * fastest block, and the fastest candidate is kept.  The blocks are real
 * steps of the simulation: it first steps to a block boundary (0 to 63
 * steps), then rounds x 12 x 64 steps (14 on a grid that takes the fused
 * pass); report->steps counts both.  `report`
 * may be NULL.  Synchronises.  Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
int pic_tune(pic_handle *h, int32_t rounds, pic_tune_report *report);

/* ---------------------------------------------------------------- batch --
 * Several independent simulations (same device, any sizes and precisions)
 * stepped together.  The paper has no counterpart; it serves parameter sweeps
 * (films of different thicknesses, bunches of different energies): every
 * whole block of 64 steps of every instance is captured into one CUDA graph,
 * so instances too small to fill the GPU share it instead of running one
 * after another.  Instances whose grids take the fused field pass (two or
 * more of them, pic_stats.field_path 1) step together: per step ONE joint
 * field pass whose work items (tiles x plane chunks) are those of all of
 * them, launched once per tile kind, beside each one's push, deposit and
 * sources on its own streams, then each one's free-current correction and
 * probe sample.  The other instances run their blocks as branches of their own on
 * their own streams.  The arithmetic of each instance is that of pic_step
 * (see pic_batch_set_joint for the rounding of the joint pass). */
typedef struct pic_batch pic_batch;

/* Group n handles (not owned; each must outlive the batch and appear once).
 * stream: the CUDA stream the batch graph is launched on (NULL: the batch
 * creates its own).  Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
int pic_batch_create(int n, pic_handle *const *handles, void *stream, pic_batch **out);

/* Advance every instance by nsteps.  While every instance sits at a 64-step
 * block boundary (no probe samples buffered), whole blocks go through the
 * batch graph; the rest run per instance as pic_step does.  The graph is
 * captured again when an instance changed in a way that invalidates captured
 * steps (particles added, deposit switched, sources or stream changed).
 * Asynchronous; each instance's stream is ordered after the batch, so its own
 * calls (pic_probe_read, pic_get_field, ...) see the result.  Errors:
 * PIC_ERR_ARG, PIC_ERR_CUDA. */
int pic_batch_step(pic_batch *b, int64_t nsteps);

/* Wait for the batch and every instance; reports device errors as pic_sync. */
int pic_batch_sync(pic_batch *b);

/* How many instances run side by side in the batch graph: the instances are
 * dealt, largest first, to `lanes` chains (each to the chain with the fewest
 * cells so far); the chains run side by side and the instances of a chain
 * one after another.  0 (the default): every instance beside every other.
 * Grids that fill the GPU alone can lose L2 locality when all run at once.
 * Errors: PIC_ERR_ARG. */
int pic_batch_set_lanes(pic_batch *b, int32_t lanes);

/* joint = 1 (the default): the fused passes of the instances that take one
 * run as one joint pass per step (above; its work items are runs of 32
 * planes of a tile column, longer than an instance alone uses, since the
 * joint pass has items enough to fill the GPU); 0: every instance runs its
 * blocks as a branch of its own.  The results agree to FP32 rounding (the
 * joint kernels are compiled separately, and the compiler may contract
 * products and sums into FMAs differently).  Errors: PIC_ERR_ARG (joint not
 * 0 or 1). */
int pic_batch_set_joint(pic_batch *b, int32_t joint);

/* pic_tune for the batch as a whole: each candidate is applied to every
 * instance and timed on whole batch blocks (the box candidates at the first
 * instance's sort interval, with the fused pass wherever an instance's grid
 * takes it), then field_path {1, 0}, then the lanes {1, 2, 4, 8, all} (those
 * below the instance count) with the best settings; the fastest settings are
 * applied to every instance and the fastest lanes to the batch.  Instances
 * not at a block boundary first step to it on their own (up to 63 steps
 * each); then every instance advances by report->steps = rounds x (14 +
 * lane candidates) x 64 steps.  `report` may be NULL.  Synchronises.  Errors:
 * PIC_ERR_ARG, PIC_ERR_CUDA. */
int pic_batch_tune(pic_batch *b, int32_t rounds, pic_tune_report *report);

/* Release the batch (not its instances).  NULL is accepted. */
int pic_batch_destroy(pic_batch *b);

/* Probe-DFT fold that allocates no device memory.  The paper has no
 * counterpart; this is a service for callers that cannot call cudaMalloc:
 * code whose device memory is owned entirely by another allocator (a
 * framework's caching pool, a fixed arena budgeted at start-up) and
 * latency-critical loops where cudaMalloc/cudaFree would synchronise the
 * device.  It does what pic_probe_read's flush does for a handle, on
 * caller-provided device arrays:
 *   F[p][c][f] += dt * sum_s samples[s][p][c] * exp(+i 2 pi freq_hz[f] (first_step+s+1) dt)
 * for s < count and the components c set in comp_mask (FP64 throughout).
 * samples: device [count][np][3] (sample s is E at step first_step+s+1);
 * freq_hz: device [nf]; F: device [np][3][nf][2] (re, im), accumulated into.
 * The caller owns all three arrays.  The phase table lives in a fixed 2 MiB
 * __device__ array inside the library (held on every GPU that loads the
 * library until the process exits); nf above 2048 is rejected with
 * PIC_ERR_ARG.  The first call on each device looks up that array's device
 * address with the device current (and again after a reset of the device
 * gives it a new context); make that first call before any stream capture.  Every call on a device shares the array, so calls whose work
 * overlaps on the GPU (different streams, or threads) race on it; serialise
 * them on one stream.  Asynchronous on `stream` (NULL: the legacy default
 * stream); launch errors are returned, kernel faults surface at the next
 * synchronisation. */
int pic_dft_fold_static(const double *samples, int64_t count, int np, uint32_t comp_mask,
                        const double *freq_hz, int nf, int64_t first_step, double dt, double *F,
                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
