/*
 * lc.h -- C ABI of liblc, the GB300 (sm_103a) light-cone retarded-field library.
 *
 * The library computes the time-delayed ("retarded", light-cone) radiation
 * field of Ahn 2015 (arXiv:1502.02294), e.g. the Lyman-Werner background:
 *
 *   J(x, tau_obs) = U * sum_n  G_n (*) f_n                       (Eq. 9-11)
 *
 * where f_n is the gridded source luminosity of past slice n (Eq. 17 source
 * term, l^3 absorbed as in Eq. 11), G_n the effective periodic retarded
 * Green's function of the shell that slice occupies on the observer's past
 * light cone (Eq. 10, LW kernel of Eqs. 14-17), and (*) a periodic
 * convolution evaluated with the convolution theorem (Eqs. 12-13):
 *
 *   Jhat(k) = sum_n Ghat_n(k) fhat_n(k),    J = U * IDFT(Jhat)  (1/N^3 per Eq. 12)
 *
 * The steps of Section 2.2 map onto the calls:  steps 1-3 (slicing, Green's
 * functions by direct summation over periodic unit-source images, their
 * transforms, precomputed per observing time as the paragraph after the
 * algorithm suggests) -> lc_plan_create / lc_plan_prepare;  step 4 (transform
 * of the source term) -> lc_push_sources;  steps 5-6 (products, inverse
 * transform, sum over slices; the sum is taken in k-space, which is exact by
 * linearity, so one inverse transform suffices) -> lc_retarded_field.
 *
 * Conventions common to every call:
 *   - Units: comoving Mpc for lengths; luminosities in any unit; J comes out
 *     in (luminosity unit) / Mpc^2 / sr times out_unit.
 *   - Grids are C order, index (i, j, k) at flat position (i*N + j)*N + k, the
 *     cell of index i centred at x = i*l, l = L/N (Section 2.2).
 *   - Pointers may be host or device memory (detected with
 *     cudaPointerGetAttributes); the caller owns them and the library copies
 *     what it needs.  All device work runs on the plan's stream.
 *   - Every call returns an lc_status.  LC_OK is 0.  Argument errors leave
 *     the plan usable; LC_ERR_CUDA and LC_ERR_TIMEOUT mark the plan failed
 *     (every later call on it returns LC_ERR_CUDA).
 *   - There is no CPU fallback: without a usable CUDA device the calls
 *     return LC_ERR_CUDA.
 */
#ifndef LC_H
#define LC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lc_plan lc_plan; /* opaque, owned by the library */
typedef struct lc_step_graph lc_step_graph;

typedef enum {
    LC_OK = 0,
    LC_ERR_INVALID_ARG = 1,      /* a null pointer, a bad value, a non-finite or negative luminosity */
    LC_ERR_UNSUPPORTED_SIZE = 2, /* N not in {8,16,32,64,96,128,192,256,384,512}, or a table too large */
    LC_ERR_STEP_ORDER = 3,       /* push not strictly increasing, or field for a step that is not the last pushed */
    LC_ERR_OOM = 4,              /* device allocation failed (plan left usable, nothing allocated) */
    LC_ERR_CUDA = 5,             /* a CUDA runtime error; the plan is marked failed */
    LC_ERR_TIMEOUT = 6,          /* a bounded device wait gave up; the plan is marked failed */
    LC_ERR_DEVICE_CHECK = 7      /* a device-side input check failed (reported by lc_plan_check) */
} lc_status;

/* Flat LCDM, no radiation: H(z) = 100 h sqrt(omega_m (1+z)^3 + 1 - omega_m) km/s/Mpc. */
typedef struct {
    double omega_m;
    double h;
} lc_cosmology;

enum { LC_STEPS_EXPLICIT = 0, LC_STEPS_EQUAL_TIME = 1, LC_STEPS_EQUAL_TAU = 2 };
enum { LC_HISTORY_FP32 = 0, LC_HISTORY_BF16 = 1 };

/* The radial kernel: the dilution factor F(|x - x'|, tau, tau') of the
 * generic retarded Green's function (Eq. 7), which the method needs only as
 * a function of distance (with tau' fixed by the light cone).
 *   LC_KERNEL_LW:  the Lyman-Werner kernel, Eqs. 14-17:
 *                  g(r) = (1+z)^3 f_mod(r) / ((4 pi)^2 (1+z_s) r^2), f_mod of
 *                  Eq. 15 with alpha(z_s) of Eq. 16; horizon r / alpha = 97.39.
 *   LC_KERNEL_EXP: the same dilution and redshift factors with a
 *                  distance-only attenuation in place of f_mod:
 *                  g(r) = (1+z)^3 exp(-r / lambda) / ((4 pi)^2 (1+z_s) r^2)
 *                  for r < r_max, 0 beyond; r_max is this kernel's horizon
 *                  (lambda = kernel_length, r_max = kernel_rmax, comoving Mpc). */
enum { LC_KERNEL_LW = 0, LC_KERNEL_EXP = 1 };

/* The near field of the innermost slice.  The 5^3 cells around each source's
 * cell (each of its 8 cells with the cloud-in-cell deposit) are taken out of
 * the FFT path of the innermost shell and added per source in FP64, so the
 * largest Green's-function values never pass through FP32 (or BF16) spectra:
 *   LC_NEAR_NGP:     with the source at its cell centre (the grid Green's
 *                    function itself, so the field is exactly Eq. 11);
 *   LC_NEAR_SUBCELL: from the source's own position, the particle-mesh hybrid
 *                    that the Discussion suggests for sources resolved below
 *                    the mesh: each target cell gets the s^3 sub-sample average
 *                    of g around the source (over the periodic images, inside
 *                    the innermost shell and the horizon) times the shell's
 *                    normalisation factor.  Needs the NGP deposit (either
 *                    history);
 *   LC_NEAR_NONE:    no split: the innermost shell goes through the FFT path
 *                    whole (no per-source near-field work). */
enum { LC_NEAR_NGP = 0, LC_NEAR_SUBCELL = 1, LC_NEAR_NONE = 2 };

/* How a source's luminosity is assigned to the grid (the source term f_n of
 * Eq. 11 and Eq. 17, l^3 absorbed), in integer fixed point either way: a unit
 * S = 2^(E-62) with n_src * max(lum) < 2^E, q = rint(lum / S) per source, and
 * int64 sums per cell, so the grid is bit-exact and independent of source
 * order.
 *   LC_DEPOSIT_NGP: all of q to the nearest cell centre,
 *                   i = floor(x / l + 1/2) mod N per axis;
 *   LC_DEPOSIT_CIC: cloud in cell: along each axis the two cell centres
 *                   around the source, i0 = floor(x / l) and i0 + 1 (mod N),
 *                   with weights 1 - f and f, f = x / l - i0; q is split along
 *                   x, each part along y, each of those along z, the upper
 *                   part of a split being min(q', rint(q' f)) and the lower
 *                   the rest, so the 8 integer shares sum to q exactly. */
enum { LC_DEPOSIT_NGP = 0, LC_DEPOSIT_CIC = 1 };

/* Which horizon the Lyman-Werner kernel is cut at (LC_KERNEL_LW only).
 *   LC_HORIZON_EQ15:  f_mod of Eq. 15, zero where r / alpha(z_s) > 97.39;
 *   LC_HORIZON_ROUGH: the rough horizon of Section 1, r <= 100 [21 / (1 + z_s)]^0.5
 *                     Mpc, with z the emission redshift z_s; inside it f_mod of
 *                     Eq. 15 without its cut, clamped at 0 (it turns negative at
 *                     r / alpha = 116.29 ln(1.7 / 0.7)^(1 / 0.68), about 97.54). */
enum { LC_HORIZON_EQ15 = 0, LC_HORIZON_ROUGH = 1 };

/* How time is sliced (step 1 of Section 2.2) and how the field is evaluated.
 * Step s spans [tau_s, tau_{s+1}] and is observed at its end, tau_{s+1}; the
 * sources pushed at step s stand for the source term frozen over that step
 * (Eq. 9).  Slice n seen from step s occupies the half-open shell
 * [tau_{s+1} - tau_{n+1}, tau_{s+1} - tau_n) and counts while its inner radius
 * is inside the kernel's horizon r_h (for the LW kernel the radius where
 * r / alpha(z_s(r)) = 97.39, Eqs. 15-16). */
typedef struct {
    int n_steps;           /* number of steps (>= 1) */
    int spacing;           /* LC_STEPS_* */
    const double* z_edges; /* LC_STEPS_EXPLICIT: n_steps + 1 decreasing redshifts (copied) */
    double z_start;        /* LC_STEPS_EQUAL_TIME: first edge (highest z) */
    double z_end;          /* EQUAL_TIME and EQUAL_TAU: last edge */
    int n_shell;           /* LC_STEPS_EQUAL_TAU: step width r_h(z_end) / n_shell in conformal time (r_h: the kernel's horizon) */
    int subsamples;        /* s: sub-cell samples per axis in G_n (even, 2..16; 0 -> 4) */
    int history;           /* LC_HISTORY_FP32, or LC_HISTORY_BF16 (spectra stored / DC, scale kept in FP32) */
    int normalise;         /* 1: scale each G_n so that l^3 sum G_n = int 4 pi r^2 g dr over its shell */
    double out_unit;       /* U: multiplies J (0 -> 1) */
    int kernel;            /* LC_KERNEL_LW (0, default) or LC_KERNEL_EXP */
    double kernel_length;  /* LC_KERNEL_EXP: attenuation length lambda > 0, comoving Mpc */
    double kernel_rmax;    /* LC_KERNEL_EXP: cut-off radius r_max > 0, comoving Mpc */
    int near_mode;         /* LC_NEAR_NGP (0, default), LC_NEAR_SUBCELL (FP32 history, NGP deposit) or LC_NEAR_NONE */
    int deposit;           /* LC_DEPOSIT_NGP (0, default) or LC_DEPOSIT_CIC */
    int horizon_mode;      /* LC_HORIZON_EQ15 (0, default) or LC_HORIZON_ROUGH (LW kernel only) */
    int n_shell_max;       /* > 0: at most this many lookback slices per observing step (the newest
                              ones; the number of stored Green's functions per observing time, which the
                              paragraph after the algorithm of Section 2.2 lets vary); 0: no cap */
} lc_steps;

/* Create a plan for an N^3 periodic grid of side box_mpc.
 * N in {8, 16, 32, 64, 96, 128, 192, 256, 384, 512}.  cuda_stream may be NULL
 * (default stream) or a cudaStream_t.  Allocates the device history ring,
 * work buffers and tables; Green's function tables are built lazily per
 * observing step (or eagerly with lc_plan_prepare).  On error *out is NULL. */
lc_status lc_plan_create(int n, double box_mpc, const lc_cosmology* cosmo, const lc_steps* steps,
                         void* cuda_stream, lc_plan** out);

/* Build (precompute) the Green's function tables of observing steps
 * [step_begin, step_end) -- steps 2-3 of Section 2.2 and the stored
 * "data files" of the paragraph after it.  Idempotent. */
lc_status lc_plan_prepare(lc_plan* plan, int step_begin, int step_end);

/* Deposit the sources active during step `step` (nearest grid point or cloud
 * in cell, lc_steps.deposit; integer fixed point: bit-exact and independent of
 * source order) and transform them into the history ring (step 4 of
 * Section 2.2).
 *   pos: n_src * 3 doubles (x, y, z in comoving Mpc, any real value; wrapped
 *        periodically), host or device.
 *   lum: n_src doubles, finite and >= 0, host or device.
 * Steps must strictly increase; a step that is never pushed counts as having
 * no sources.  Host inputs are validated here (LC_ERR_INVALID_ARG); device
 * inputs are validated on the device and reported by lc_plan_check. */
lc_status lc_push_sources(lc_plan* plan, int step, int64_t n_src, const double* pos, const double* lum);

/* The retarded field at the end of step `step` (steps 5-6 of Section 2.2),
 * which must be the last pushed step.  out: N^3 floats, C order, host or
 * device.  With a host `out` the call waits for the result; with a device
 * `out` it only enqueues work on the plan's stream. */
lc_status lc_retarded_field(lc_plan* plan, int step, float* out);

/* lc_retarded_field without the wait: the same field of the same step (same
 * rules), but with a host `out` the call returns once the work and the
 * device-to-host copy are enqueued, and *ticket (> 0) names that copy.  The
 * copy runs on a copy stream of the plan, out of one of two device stages,
 * so the next steps' pushes and fields compute while it drains (into
 * page-locked memory by a small copy kernel writing through the buffer's
 * device view, LC_D2H_CTAS CTAs, default 8; LC_D2H=ce in the environment
 * uses the copy engine); `out` holds
 * the field once lc_plan_wait(plan, *ticket) returns, and must stay valid
 * until then (page-locked host memory makes the copy asynchronous; with
 * pageable memory the call itself waits for the copy).  With a device `out`
 * this is lc_retarded_field and *ticket = 0.
 * Errors: LC_ERR_INVALID_ARG for ticket == NULL or a host `out` inside a
 * graph capture, otherwise those of lc_retarded_field. */
lc_status lc_retarded_field_async(lc_plan* plan, int step, float* out, uint64_t* ticket);

/* Block the calling thread until the output named by `ticket` is in host
 * memory (ticket 0: until the plan's stream is idle).  Waiting on an older
 * ticket than the last is allowed; a ticket never issued is
 * LC_ERR_INVALID_ARG. */
lc_status lc_plan_wait(lc_plan* plan, uint64_t ticket);

/* lc_plan_wait without blocking: *done = 1 if the output named by `ticket`
 * is in host memory (ticket 0: the plan's stream is idle), else 0.  Each
 * ticket has its own completion event for the next 16 tickets; a ticket
 * older than that reports done once a later copy has finished (copies of a
 * plan complete in ticket order; never early).  Same errors as
 * lc_plan_wait. */
lc_status lc_plan_poll(lc_plan* plan, uint64_t ticket, int* done);

/* The same field computed "instantaneously" (action at a distance, Eq. 18 of
 * Section 3): every shell's Green's function is applied to the sources of
 * step `step` itself, i.e. the source distribution frozen at the observing
 * redshift, with all other factors (dilution, (1+z)^3/(1+z_s), f_mod, the
 * light-travel radius of each shell) kept.  The fractional difference
 * (J_instant - J) / J is the paper's f_diff.  Same arguments and rules as
 * lc_retarded_field. */
lc_status lc_instant_field(lc_plan* plan, int step, float* out);

/* Forget the history (ring) so that steps can start again at 0; the Green's
 * function tables are kept. */
lc_status lc_plan_reset(lc_plan* plan);

/* Synchronise the plan's stream and report device-side input checks
 * (LC_ERR_DEVICE_CHECK) and CUDA errors. */
lc_status lc_plan_check(lc_plan* plan);

lc_status lc_plan_set_stream(lc_plan* plan, void* cuda_stream);
lc_status lc_plan_destroy(lc_plan* plan);
const char* lc_status_string(lc_status status);

/* Green's-function table budget.  The paper precomputes one Ghat table per
 * observing step (the paragraph after the algorithm of Section 2.2); over a
 * long run the tables of all steps can exceed device memory.  With a budget
 * of `bytes` (0, the default: no limit), building the table of a step first
 * frees tables of other steps, earlier ones oldest first, then later ones
 * latest first, until the total fits; a freed table is rebuilt, identically,
 * if its step is evaluated again.  Tables captured in a graph are never
 * freed (step graphs: until the graph is destroyed; batch graphs: for the
 * life of the plan), so the budget is soft.  lc_plan_table_bytes: the bytes
 * the plan's tables hold now. */
lc_status lc_plan_set_table_budget(lc_plan* plan, size_t bytes);
size_t lc_plan_table_bytes(const lc_plan* plan);

/* Device bytes held by the plan (ring + tables + buffers), for HBM-budget admission. */
size_t lc_plan_device_bytes(const lc_plan* plan);

/* Bytes lc_plan_create would allocate before any Green's function table
 * (ring, buffers), and the bytes of one observing step's table.  Host only. */
lc_status lc_plan_estimate(int n, const lc_steps* steps, const lc_cosmology* cosmo, size_t* base_bytes,
                           size_t* table_bytes_per_step);

/* Geometry of observing step `step`: number of active slices, their shell
 * radii (lookback j = 0 is the newest slice) and the horizon.  Arrays of at
 * least step + 1 entries, or NULL. */
lc_status lc_step_shells(const lc_plan* plan, int step, int* n_active, double* r_lo, double* r_hi, double* r_h,
                         double* shell_integral);

/* Ring depth and other plan facts. */
typedef struct {
    int n;
    int n_steps;
    int n_ring;            /* history slots = max active slices over all steps */
    int history;
    int wedge_size;        /* C(N/2 + 3, 3) */
    int spectrum_row;      /* padded complex row length of the half spectrum */
    double box_mpc;
    const double* z_edges; /* n_steps + 1 entries, owned by the plan */
} lc_plan_info_t;
lc_status lc_plan_info(const lc_plan* plan, lc_plan_info_t* info);

/* Ghat_j of observing step `step` on the symmetric wedge 0 <= p <= q <= r <= N/2
 * (index C(r+2,3) + C(q+1,2) + p; Ghat is real and invariant under sign flips
 * and permutations of (p, q, r)), building the step's table if needed.
 * out: wedge_size floats, host or device.  Also returns Ghat_j(0) in FP64. */
lc_status lc_plan_green_wedge(lc_plan* plan, int step, int lookback, float* out, double* ghat0);

/* Batched evaluation: for every i, push plans[i]'s sources for steps[i] (if
 * n_src[i] >= 0) and compute its retarded field into outs[i] (device
 * pointers), with all instances' kernels launched phase by phase on the
 * stream of plans[0] so that uneven instances overlap on the device. */
lc_status lc_batch_step(lc_plan* const* plans, int n, const int* steps, const int64_t* n_src,
                        const double* const* pos, const double* const* lum, float* const* outs);

/* --- checkpoint / resume ---------------------------------------------------------- */

/* The state a plan carries from step to step is the history of past source
 * spectra that the retarded sum of Eq. 11 reads (one slice per active shell),
 * with each slice's fixed-point unit and exact total, the last pushed step,
 * and the innermost slice's source cells (near field).  The
 * Green's function tables are not part of it: they are a deterministic
 * function of the plan's parameters and are rebuilt on demand.
 *
 * lc_plan_checkpoint_bytes: size of that state in bytes (a 256-byte header,
 * the per-slot arrays, the near-field list, then the ring).
 * lc_plan_save: writes it to buf (host or device memory, `size` >= that many
 * bytes); returns after the copy has completed.  The header records N, the
 * step count, ring depth, history precision and a 64-bit hash of every
 * parameter that defines the method (box, cosmology, step edges, subsamples,
 * normalisation, output unit).
 * lc_plan_load: restores a checkpoint into a plan created with the same
 * parameters (LC_ERR_INVALID_ARG if the header, hash or size does not match,
 * leaving the plan unchanged); the next push must be for a later step than
 * the saved one.  Both synchronise the plan's stream. */
size_t lc_plan_checkpoint_bytes(const lc_plan* plan);
lc_status lc_plan_save(lc_plan* plan, void* buf, size_t size);
lc_status lc_plan_load(lc_plan* plan, const void* buf, size_t size);

/* --- CUDA graphs of whole steps ------------------------------------------------ */

/* One observing step captured as a CUDA graph: lc_push_sources(step, ...) then
 * lc_retarded_field(step, out), replayed by lc_graph_launch with one launch
 * call (the kernels of steps 4-6 of Section 2.2 back to back on the device).
 * pos, lum and out are DEVICE pointers, read and written at every replay;
 * the step's Green's function table is built before capture.  The plan must
 * not be captured concurrently from another thread. */
lc_status lc_graph_create(lc_plan* plan, int step, int64_t n_src, const double* pos, const double* lum, float* out,
                          lc_step_graph** graph);
/* Replay on the plan's stream.  Same ordering rule as lc_push_sources: the
 * step must be later than the last pushed step; it becomes the last pushed. */
lc_status lc_graph_launch(lc_step_graph* graph);
lc_status lc_graph_destroy(lc_step_graph* graph);

/* Many uneven instances (plans of different N, shell counts and source
 * counts), one observing step each, captured as ONE CUDA graph: every
 * instance's push + field is a parallel branch, so the instances overlap on
 * the device and the whole batch is one launch.  Arguments are arrays of n
 * (a plan at most once); pointers are device pointers, read/written at every
 * replay.  Launch on `cuda_stream` (NULL: the default stream); each plan's
 * steps must increase across launches as for lc_push_sources. */
typedef struct lc_batch_graph lc_batch_graph;
lc_status lc_batch_graph_create(lc_plan* const* plans, int n, const int* steps, const int64_t* n_src,
                                const double* const* pos, const double* const* lum, float* const* outs,
                                lc_batch_graph** graph);
lc_status lc_batch_graph_launch(lc_batch_graph* graph, void* cuda_stream);
lc_status lc_batch_graph_destroy(lc_batch_graph* graph);

/* --- tracing ------------------------------------------------------------------ */

/* Phases of one step, each timed with a pair of CUDA events on the plan's
 * stream when timing is enabled.  Where plane kernels do z and y together
 * (N <= 192, and 256 in the cluster form), LC_PHASE_R2C_Z and LC_PHASE_C2R_Z
 * hold both passes and the y phases stay empty; where a short near-field list
 * runs on extra CTAs of the inverse plane kernel, its scatter counts in
 * LC_PHASE_C2R_Z and LC_PHASE_NEAR holds the fold alone. */
enum {
    LC_PHASE_DEPOSIT = 0,    /* zero grid + source checks + fixed-point deposit */
    LC_PHASE_R2C_Z = 1,      /* z rows, real -> complex (int64 prologue) */
    LC_PHASE_FWD_Y = 2,      /* y pass, forward */
    LC_PHASE_FWD_X_RING = 3, /* x pass, forward, into the history ring slot */
    LC_PHASE_MAC_X = 4,      /* shell multiply-accumulate fused with the inverse x pass */
    LC_PHASE_INV_Y = 5,      /* y pass, inverse */
    LC_PHASE_C2R_Z = 6,      /* z rows, complex -> real, scaled output */
    LC_PHASE_NEAR = 7,       /* innermost shell's near cube, exact FP64 scatter + fold */
    LC_N_PHASES = 8
};
/* Enable (1) or disable (0) per-phase event timing on this plan. */
lc_status lc_plan_set_timing(lc_plan* plan, int enable);
/* Synchronise and return the accumulated milliseconds and launch counts per
 * phase (arrays of LC_N_PHASES, either may be NULL); reset != 0 clears them. */
lc_status lc_plan_timing(lc_plan* plan, double* ms, int64_t* launches, int reset);
/* Number of kernels this library has launched in this process (all plans and
 * stand-alone calls). */
uint64_t lc_kernel_launches(void);

/* --- autotuning ---------------------------------------------------------------- */

/* The shell multiply-accumulate runs in one of four kernels: a register-gather
 * pass (gather), a bulk-copy pipelined kernel over the full tiles plus the
 * gather pass for the Nyquist tiles (bulk), and a warp-specialised kernel
 * over every tile, one tile per CTA (ws) or the tiles of lines q and N - q
 * together (ws2).  Each plan times every kernel built for its grid on its own
 * buffers when it first builds a table for a new (device, N, history, active
 * slices) combination (seven launches, each after an L2 flush) and keeps the
 * one with the lowest median.  Choices are shared by all plans
 * of the process and persisted to the file named by the environment variable
 * LC_AUTOTUNE_CACHE if set; LC_MAC_VARIANT=gather|bulk|ws|ws2 forces one
 * kernel where it is built.  This writes the current choices ("key variant"
 * lines) into buf (size bytes, NUL-terminated) and returns the full length. */
int lc_autotune_report(char* buf, int size);

/* The FFT passes of Eq. 12 along y and x (and along z) come in five kernel
 * forms for N = 256, 384 and 512: LC_FFT_STAGES, block-wide Stockham radix stages
 * in shared memory (every N), and four forms with one lane per tile column
 * (a lane group per row pair along z), the 16-point DFTs in registers and a
 * single shared-memory exchange between the two radix stages:
 * LC_FFT_LANES (tiles copied by 16-byte asynchronous copies into four
 * stages, one CTA per SM), LC_FFT_LANES3 (three stages, two CTAs per SM),
 * LC_FFT_TMA (tiles moved by tensor-map TMA, three stages, two CTAs per SM)
 * and LC_FFT_TMA4 (TMA, four stages, one CTA per SM).  Grids with plane
 * kernels (N = 32 ... 192: z and y per x-plane in one kernel) have two:
 * LC_FFT_STAGES (staged plane kernels) and LC_FFT_LANES (the transforms in
 * registers, one shared-memory exchange per axis); 8 and 16 have one.
 * N = 256 has a sixth, LC_FFT_PLANE4: the z and y passes of a step in one
 * kernel each way, an x-plane per cluster of four CTAs (two per SM), each
 * holding a quarter of the plane's columns (the z pass of its quarter of
 * the rows stores into every CTA's shared memory), the x passes as
 * LC_FFT_LANES.
 * The first plan created for a grid size times every form on its own
 * buffers (forward and inverse passes of one step, each launch after an L2
 * flush, median of seven) and keeps the fastest
 * for the rest of the process (the choice is listed by lc_autotune_report
 * and persisted with the shell-MAC choices);
 * LC_FFT_VARIANT=stages|lanes|lanes3|tma|tma4|plane4 forces one.
 * lc_fft_set_variant(n, v) forces v for grid size n from now on (later plans
 * and stand-alone calls; a table already built keeps its values), and
 * lc_fft_variant(n) returns the form in use (-1: n not supported).
 * LC_ERR_UNSUPPORTED_SIZE if n has no such form. */
enum {
    LC_FFT_STAGES = 0,
    LC_FFT_LANES = 1,
    LC_FFT_LANES3 = 2,
    LC_FFT_TMA = 3,
    LC_FFT_TMA4 = 4,
    LC_FFT_PLANE4 = 5
};
lc_status lc_fft_set_variant(int n, int variant);
int lc_fft_variant(int n);

/* --- light-cone vs instantaneous field ------------------------------------------ */

/* The fractional difference f_diff = (J_instant - J) / J that Section 3 uses
 * (after Eq. 18) to measure the light-cone effect, per cell, from a field of
 * lc_retarded_field and one of lc_instant_field for the same step.  All
 * three arrays hold n floats in device memory (LC_ERR_INVALID_ARG
 * otherwise); the difference and quotient are taken in FP64 and rounded
 * once.  Cells where both fields are 0 get 0; where only J is 0, IEEE
 * +-infinity.  Asynchronous on `stream`. */
lc_status lc_fdiff_map(int64_t n, const float* j_retarded, const float* j_instant, float* out, void* stream);

/* --- the hot-path kernels as stand-alone calls (tests, users) --------------- */

/* The fixed-point deposit of lc_push_sources on its own: scale S = 2^(E-62)
 * with n_src * max(lum) < 2^E, q = rint(lum / S), grid[cell] = sum of the
 * shares (int64, N^3, device or host), *total = sum q.  deposit:
 * LC_DEPOSIT_NGP (cell = floor(x / l + 1/2) mod N per axis) or LC_DEPOSIT_CIC
 * (the 8 shares of each q described with LC_DEPOSIT_CIC).  Synchronises the
 * stream; LC_ERR_DEVICE_CHECK if a source was invalid (it is left out). */
lc_status lc_deposit_grid(int n, double box_mpc, int deposit, int64_t n_src, const double* pos, const double* lum,
                          int64_t* grid, double* scale, int64_t* total, void* cuda_stream);

/* 3D real-to-complex DFT with the forward sign of Eq. 12 (e^{-2 pi i k.x / N},
 * unnormalised): in N^3 floats, out N*N*(N/2+1) complex floats (interleaved),
 * C order, device pointers. */
lc_status lc_fft_r2c(int n, const float* in, float* out_complex, void* cuda_stream);

/* Inverse of Eq. 12 (e^{+2 pi i k.x / N}), times `scale` (pass 1/N^3 for the
 * exact inverse): in N*N*(N/2+1) complex floats, out N^3 floats, device pointers. */
lc_status lc_fft_c2r(int n, const float* in_complex, float* out, float scale, void* cuda_stream);

/* lc_fft_r2c without any device allocation (the paper has no counterpart:
 * this is a library-usage variant).  For callers that cannot call cudaMalloc
 * (a device memory pool that owns all memory, a host application that
 * forbids allocation, or a loop that must not synchronise on one), the work
 * spectrum and twiddle table live in one static 4 MiB device array that the
 * library reserves on every GPU it is used on until the process exits.
 *   n: 8, 16, 32, 64 or 96 (larger grids do not fit: LC_ERR_UNSUPPORTED_SIZE).
 *   in, out_complex: device pointers as for lc_fft_r2c.
 * The work is only enqueued on cuda_stream (no synchronisation).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress),
 * and so does the first call in each new context of the device (after
 * cudaDeviceReset); make that first call before capturing a stream.  All calls
 * share the one array: calls queued one after another on one stream are
 * ordered and safe, but calls whose work may overlap on the GPU (different
 * streams without ordering) race and must not be issued. */
lc_status lc_fft_r2c_static(int n, const float* in, float* out_complex, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LC_H */
