/*
 * sbp.h — C ABI of the GB300 shearing-box Poisson solver (VGF-HybridBC).
 *
 * Solves ∇²Φ = 4πGρ (arXiv 2510.10070, Eq. Poisson) on a Cartesian box with
 * shear-periodic horizontal and vacuum vertical boundary conditions, by the
 * discrete-Green's-function spectral method of Sect. 2.3:
 *
 *   Φ = 4πG F⁻¹( Ĝ^L(k(t), k_z) · F(ρ zero-padded to 2·nz in z) ),
 *
 * truncated back to the physical cells, where F is the 3D DFT, k(t) is the
 * sheared horizontal wave-vector of Sect. 2.1 and Ĝ^L is Eq. (Green's
 * function regularized in Fourier) with L = Lz.  The density is taken in the
 * periodic (remapped) frame at shear time t and the potential is returned in
 * the same frame (step 2 of the three-step scheme of Sect. 2.1).
 *
 * Conventions used by every call:
 *   - rho and phi are DEVICE pointers to dense C-order arrays [nz][ny][nx]
 *     (x fastest) of double (SBP_F64) or float (every other dtype).
 *   - Cells are cell-centred; the vertical window is [-Lz/2, Lz/2].
 *   - The output is the real part of the complex solve, i.e. the multiplier
 *     is ½[Ĝ(k) + Ĝ(k of the Hermitian partner)], which differs from Ĝ only
 *     on the Nyquist planes of a sheared box.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Every call is asynchronous on that stream; the caller synchronises.
 *   - Nothing here calls exit() or traps: failures come back as sbp_status.
 *
 * Ownership: the caller owns rho and phi.  A plan owns its device workspace
 * (the half spectrum, (nx/2+1)·ny·nz complex values, plus small tables), which
 * it allocates in sbp_plan_create and frees in sbp_plan_destroy.  One solve
 * may be in flight per plan; use one plan per stream.
 */
#ifndef SBP_H
#define SBP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbp_plan_s* sbp_plan;

/* Arithmetic of the FFT passes.  SBP_F64: everything in FP64.  SBP_F32: FP32
 * passes; FP64 Green's parameters, FP64-derived twiddles, and an FP64 k = 0
 * (mean-mode) side path.  The split dtypes are reserved for tensor-core
 * radix stages and are rejected with SBP_ERR_UNSUPPORTED_DTYPE. */
typedef enum {
    SBP_F64 = 0,
    SBP_F32 = 1,
    SBP_F32_SPLIT_F16 = 2,
    SBP_F32_SPLIT_BF16 = 3
} sbp_dtype;

typedef enum {
    SBP_OK = 0,
    SBP_ERR_INVALID_ARG = 1,       /* NULL/unaligned/partially overlapping pointer, bad number */
    SBP_ERR_UNSUPPORTED_SIZE = 2,  /* a dimension outside the supported lengths */
    SBP_ERR_OUT_OF_MEMORY = 3,     /* device allocation failed */
    SBP_ERR_CUDA = 4,              /* a CUDA runtime call or kernel launch failed */
    SBP_ERR_DEVICE_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    SBP_ERR_NOT_SAME_DTYPE = 6,    /* batched call mixing dtypes */
    SBP_ERR_UNSUPPORTED_DTYPE = 7, /* dtype not built in this library */
    SBP_ERR_SCRATCH_LIMIT = 8      /* box too large for sbp_solve_noalloc's fixed workspace */
} sbp_status;

/* Plan stages that sbp_run_stage can run alone (see there). */
typedef enum {
    SBP_STAGE_X_FORWARD = 0,
    SBP_STAGE_Y_FORWARD = 1,
    SBP_STAGE_Z_CONVOLVE = 2,
    SBP_STAGE_Y_INVERSE = 3,
    SBP_STAGE_X_INVERSE = 4,
    SBP_STAGE_GREEN_TABLE = 5,
    SBP_STAGE_GREEN_FILL = 6,
    SBP_STAGE_SWEEP_FORWARD = 7,
    SBP_STAGE_SWEEP_MIDDLE = 8,
    SBP_STAGE_SWEEP_INVERSE = 9
} sbp_stage;

/*
 * sbp_plan_create — validate a box, build its tables and allocate workspace.
 *
 * Sect. 2.1 and 2.3.  nx, ny: horizontal cells, each even and ≥ 4; nz ≥ 2
 * vertical cells (zero-padded to 2·nz inside the solve).  Each of nx, ny and
 * nz must be 2^a or 3·2^a, and nx, ny, nz ≤ 2048; other sizes return
 * SBP_ERR_UNSUPPORTED_SIZE.  Lx, Ly, Lz > 0: box lengths.  q, Omega: shear
 * rate q·Ω in Δy0(t) = mod(q Ω Lx t, Ly) (the paper's q is 3/2); Omega > 0,
 * q finite.  G > 0: gravitational constant.  dtype: see sbp_dtype.
 * The plan binds to the CUDA device that is current at creation.
 * On failure *out is set to NULL and nothing is leaked.
 */
sbp_status sbp_plan_create(sbp_plan* out, int nx, int ny, int nz,
                           double Lx, double Ly, double Lz,
                           double q, double Omega, double G, sbp_dtype dtype);

/*
 * sbp_solve — one solve at shear time t (finite).
 *
 * Sect. 2.3, Eq. (Green's function regularized in Fourier) and the closing
 * convolution Φ = 4πG F⁻¹(Ĝ^L·ρ̂).  rho: device input (see conventions);
 * phi: device output of the same shape and type.  phi == rho (in place) is
 * allowed; any other overlap returns SBP_ERR_INVALID_ARG.  Both pointers must
 * be 16-byte aligned.  Runs on `stream` either three kernels (the three
 * sweeps of SBP_OPT_SCHEDULE, where they apply) or five: x forward (real to
 * half spectrum), y forward, the fused padded z pass (Green's multiply),
 * y inverse, x inverse.
 */
sbp_status sbp_solve(sbp_plan p, const void* rho, void* phi, double t, void* stream);

/*
 * sbp_solve_batched — nbox independent solves on one stream.
 *
 * Each box i is solved as sbp_solve(plans[i], rho[i], phi[i], t[i]) (bit for
 * bit when both run the same schedule, see below).  All plans must share a dtype (else SBP_ERR_NOT_SAME_DTYPE)
 * and the device.  A plan may appear only once per call.  plans, rho, phi and
 * t are HOST arrays of length nbox; rho[i] and phi[i] are device pointers.
 * phi[i] == rho[i] (in place) is allowed, as in sbp_solve.  The boxes run
 * concurrently, so a box's phi must not overlap another box's rho or phi
 * (SBP_ERR_INVALID_ARG); boxes may share the same rho.
 *
 * Execution: boxes whose plans run the three sweeps (SBP_OPT_SCHEDULE) are
 * grouped by shape, and one launch per sweep covers all boxes of a group
 * through a device table of per-box descriptors; the other boxes keep their
 * own pass kernels, spread over K parallel branches.  All of it is captured
 * once into a CUDA graph, cached by the exact (plans, rho, phi) tuple; a call
 * with a cached tuple copies the nbox shear parameters to the device and
 * replays the graph on `stream`.  The first call of a tuple tunes by timing
 * candidate graphs on `stream` (it synchronises that stream): each group as
 * grouped sweeps and as per-box five-pass kernels (the faster is kept; the
 * grouped sweeps unless they are more than 2% slower), then K (and whether
 * five-pass x/y passes run in L2-sized chunks) on the whole graph, then each
 * group's schedule flipped in turn on the whole graph (kept if the batch is
 * more than 1% faster: groups share the SMs).  The
 * candidates write into temporary outputs that the call allocates and
 * frees, so the caller's buffers see exactly one solve per call.  The choice
 * is remembered for the same plans' shapes on the same GPU type, in the
 * process and, when the environment variable SBP_TUNE_CACHE names a file, in
 * that file (one line per choice, appended), so later processes skip the
 * timing.  A later tuple with the same plans and other buffers (double
 * buffering) takes the choice without timing.  The environment variables
 * SBP_BATCH_BRANCHES=K, SBP_BATCH_CHUNK=0/1 and SBP_BATCH_SCHEDULE=1/2 (five
 * passes / grouped sweeps) force the choice; SBP_TUNE_LOG=1 prints the
 * timings and the choice to stderr.  Destroying or reconfiguring any
 * plan of a tuple drops its cached graph.  With grouped boxes the result may
 * differ from sbp_solve's by rounding where a group chose the five passes
 * while sbp_solve of that plan runs the sweeps, or the reverse; each box still
 * meets the solver's accuracy.
 */
sbp_status sbp_solve_batched(int nbox, const sbp_plan* plans, const void* const* rho,
                             void* const* phi, const double* t, void* stream);

/* sbp_plan_destroy — free a plan's device memory.  NULL-safe.  Synchronises
 * the plan's device before freeing so that no in-flight solve is cut off. */
void sbp_plan_destroy(sbp_plan p);

/* sbp_status_string — static English text for a status code. */
const char* sbp_status_string(sbp_status s);

/* Plan options for sbp_plan_set_option. */
enum {
    /* Kernel variant of the fused z pass (same result, different speed):
     * 0 = automatic (the default); 1 = 8 elements per thread, even/odd padded
     * halves in one thread; 2 = 8 elements per thread, halves in two thread
     * groups; 3 = one pruned length-2nz transform per column; 4 = even/odd
     * halves in two thread groups with the default elements per thread.
     * Variants 1-3 exist for the common lengths only
     * (SBP_ERR_UNSUPPORTED_SIZE otherwise, plan unchanged). */
    SBP_OPT_Z_VARIANT = 1,
    /* How a solve runs the x and y transforms (same result, different speed):
     * 0 = automatic (the default); 1 = separate x and y passes; 2 = fused
     * plane kernels, one z-plane per thread-block cluster, sized for one CTA
     * per SM; 3 = the same sized for two CTAs per SM.  Variants 2 and 3 exist
     * for square planes of the common sizes only (SBP_ERR_UNSUPPORTED_SIZE
     * otherwise, plan unchanged). */
    SBP_OPT_XY_PASSES = 2,
    /* 0 = the y passes load their column tiles with TMA bulk-tensor copies on
     * an mbarrier where available (the default); 1 = plain per-thread loads. */
    SBP_OPT_Y_TMA = 3,
    /* Clock cycles a kernel may wait for an asynchronous copy before it gives
     * up, records the timeout in the plan's status word and returns
     * (default 2e9, about one second).  A block whose copy was issued but is
     * late waits once more, for the same budget, before it returns, so that
     * the copy cannot land in shared memory given to another block.  After
     * SBP_ERR_DEVICE_TIMEOUT the outputs of that solve are undefined; if the
     * copy was still missing after the second wait, so are the outputs of
     * kernels that ran beside it, and the context is best torn down. */
    SBP_OPT_SPIN_BUDGET = 4,
    /* Test switch: 1 makes the TMA kernels arm no copy, so that their bounded
     * waits run out (the results are then undefined and
     * sbp_plan_sync_status reports SBP_ERR_DEVICE_TIMEOUT); 0 restores. */
    SBP_OPT_DEBUG_WITHHOLD_COPY = 5,
    /* Vertical truncation length L = alpha·Lz of the Green's function
     * (Sect. 2.3: the regularized kernel of Eq. (Green's function regularized
     * in Fourier) with L ≥ Lz; the paper takes alpha = 1.1 and pads the
     * vertical transform to 4·nz).  1 (default): L = Lz with 2·nz padding;
     * 1 < alpha ≤ 3: L = alpha·Lz with 4·nz padding (one length-4nz transform
     * per column; the periodic images then stay outside |z| < Lz).  Fourfold
     * padding is built for power-of-two nz from 32 to 512 (FP32) or 256
     * (FP64); other nz return SBP_ERR_UNSUPPORTED_SIZE and keep the old
     * setting.  SBP_OPT_Z_VARIANT then accepts only 0. */
    SBP_OPT_TRUNCATION = 6,
    /* Frame of rho and phi (Sect. 2.1, "Mapping to fully periodic points").
     * 0 (default): the periodic frame, rho~(x, y) = rho(x, y - s x) with
     * s = Delta y0 / Lx, and phi~ returned in the same frame.  1: the
     * physical (shearing) frame: the plan maps rho to the periodic frame by
     * Fourier interpolation of every x-column in y (phase exp(-i K_y s x);
     * the Nyquist row takes the real part of its phase), solves, and maps
     * phi back (phase exp(+i K_y s x)).  The mapping is fused into y
     * transforms that run before the x transforms, so a solve still makes
     * five passes.  x is the cell centre -Lx/2 + (i + 1/2) dx.  Built for nx
     * and ny in {32, 64, 96, 128, 192, 256, 512, 1024}; other sizes return
     * SBP_ERR_UNSUPPORTED_SIZE and keep the old setting.  sbp_run_stage
     * returns SBP_ERR_INVALID_ARG while it is 1. */
    SBP_OPT_FRAME = 7,
    /* Method (Sect. 2.2 and 2.3).  0 (default): VGF-HybridBC, the truncated
     * Green's function of Eq. (Green's function regularized in Fourier).
     * 1 and 2: SASHA, Phi = Phi0 + Phi_P with Phi0(z) = 4 pi G rho_mean z
     * (z/2 - zeta) for the volume-mean density and Phi_P from Eq. (Poisson
     * spectral), -4 pi G rho^/|k|^2, for rho - rho_mean zero-padded to 2 nz.
     * 1: zeta = z0 = <z rho>/<rho> as printed; 2: zeta = z0/2, the vertex that
     * cancels the uniform field -2 pi G rho_mean z0 which the 2 Lz period
     * otherwise leaves for off-centre mass.  z is the cell centre measured
     * from the box centre.  Requires SBP_OPT_TRUNCATION = 1 (else
     * SBP_ERR_UNSUPPORTED_SIZE, either order); sbp_run_stage returns
     * SBP_ERR_INVALID_ARG while it is not 0. */
    SBP_OPT_METHOD = 8,
    /* Planes per chunk of the x and y passes of sbp_solve (0, the default: the
     * whole box at once).  With chunks, the forward x and y passes run chunk
     * by chunk, and so do the inverse ones, so that a chunk's half spectrum is
     * still in L2 when the next pass reads it; fewer blocks per launch, so it
     * pays when several solves share the GPU.  sbp_solve_batched chooses by
     * itself: its first call times the graphs with and without chunks of
     * about 8 MiB of spectrum (SBP_BATCH_CHUNK=0/1 in the environment forces
     * one).  Results are identical either way. */
    SBP_OPT_XY_CHUNK = 9,
    /* Schedule of the solves (same result to rounding, different speed).
     * 0 (default): automatic; 1: five passes (x, y, z, y, x); 2: three sweeps
     * over the half spectrum, with the y transform's two radix stages fused
     * into the passes around the z pass (x + first y stage, second y stage +
     * padded z pass + first inverse y stage, second inverse y stage + x).
     * The three sweeps serve SBP_F32 plans in the periodic frame with the VGF
     * method and 2·nz padding for the box shapes built for them (nx, ny, nz)
     * = (32, 32, 32), (64, 64, 32), (64, 64, 64), (128, 128, 64),
     * (128, 128, 128), (192, 192, 96), (256, 256, 64), (256, 256, 128);
     * automatic takes them there unless a five-pass variant was asked for
     * (SBP_OPT_XY_PASSES, SBP_OPT_Z_VARIANT, SBP_OPT_Y_TMA or
     * SBP_OPT_XY_CHUNK set to a value other than 0).  2 returns
     * SBP_ERR_UNSUPPORTED_SIZE where the three sweeps do not apply.  The
     * stages of sbp_run_stage are the five-pass kernels in every schedule. */
    SBP_OPT_SCHEDULE = 10
};

/* sbp_fill_ghosts — vertical ghost layers of a solution (Sect. 2.4, last
 * paragraph: the ghost cells keep the gradient of the last active cell).
 * phi: device pointer, [nz][ny][nx] of the plan's real type (a result of
 * sbp_solve).  out: device pointer, [nz + 2 ng][ny][nx]; planes ng .. ng+nz-1
 * receive phi, and for g = 1 .. ng
 *   out[ng + nz - 1 + g] = phi[nz-1] + g (phi[nz-1] - phi[nz-2]),
 *   out[ng - g]          = phi[0]    - g (phi[1]    - phi[0]).
 * ng in [1, 16].  Both pointers 16-byte aligned and not overlapping, else
 * SBP_ERR_INVALID_ARG.  Asynchronous on `stream`.  Horizontal ghosts are the
 * caller's (periodic, or shear-periodic in the physical frame). */
sbp_status sbp_fill_ghosts(sbp_plan p, const void* phi, void* out, int ng, void* stream);

/* sbp_force — g = -grad(phi) at the cell centres by second-order central
 * differences, the force that the ghost rule of Sect. 2.4 serves.
 * phi: device pointer, [nz][ny][nx]; force: device pointer, [3][nz][ny][nx]
 * (x, y, z components).  y is periodic.  x is periodic when the plan's frame
 * (SBP_OPT_FRAME) is the periodic one; in the physical frame it is
 * shear-periodic at time t, phi(x + Lx, y) = phi(x, y + Delta y0(t)), the two
 * boundary neighbours taken by Fourier interpolation in y.  In z the ghost
 * rule makes the differences one-sided in the first and last planes.
 * Pointers 16-byte aligned and not overlapping, t finite, else
 * SBP_ERR_INVALID_ARG.  Asynchronous on `stream`. */
sbp_status sbp_force(sbp_plan p, const void* phi, void* force, double t, void* stream);

/* sbp_last_cuda_error — the CUDA runtime's message for the error behind the
 * calling thread's most recent SBP_ERR_CUDA from a kernel launch (a static
 * string; "no CUDA error recorded" if there was none).  Not part of the
 * paper's method: a diagnostic of this library. */
const char* sbp_last_cuda_error(void);

/* sbp_plan_set_option — set a plan option (see the enum above).  Unknown
 * options or values return SBP_ERR_INVALID_ARG.  Not to be called while a
 * solve of this plan is in flight.  Options that change kernels (Z_VARIANT,
 * XY_PASSES, Y_TMA, TRUNCATION) synchronise the device and drop the cached
 * sbp_solve_batched graphs that contain this plan. */
sbp_status sbp_plan_set_option(sbp_plan p, int option, double value);

/* sbp_plan_sync_status — synchronise `stream` and report device-side
 * failures of this plan's kernels since the last call: SBP_ERR_DEVICE_TIMEOUT
 * when a bounded wait gave up (the status word is then cleared), SBP_OK
 * otherwise. */
sbp_status sbp_plan_sync_status(sbp_plan p, void* stream);

/* sbp_plan_info — sizes of a plan.  Any output pointer may be NULL.
 * spectrum_pitch: complex elements per (z, y) row of the half spectrum
 * (≥ nx/2+1); workspace_bytes: device bytes the plan holds. */
sbp_status sbp_plan_info(sbp_plan p, int* nx, int* ny, int* nz, int* dtype,
                         int* spectrum_pitch, size_t* workspace_bytes);

/*
 * sbp_run_stage — run one stage of the solve alone, for stage-level tests.
 *
 * Layouts ("spectrum" = complex [nz][ny][spectrum_pitch], interleaved re/im
 * of the plan's real type, entries a ≥ nx/2+1 of each row unused):
 *   SBP_STAGE_X_FORWARD : in = real [nz][ny][nx], out = spectrum holding
 *                         X[z][y][a] = Σ_x ρ e^{-2πi a x/nx}, a ≤ nx/2.
 *   SBP_STAGE_Y_FORWARD : in = out = spectrum (in place, in must equal out);
 *                         DFT over y with e^{-2πi b y/ny}.
 *   SBP_STAGE_GREEN_FILL: in ignored, out = the spectrum buffer (unused);
 *                         fills the plan's internal Green's table for time t
 *                         (FP64 arithmetic), as the x forward pass of a solve
 *                         does.
 *   SBP_STAGE_Z_CONVOLVE: in = out = spectrum; for each column (b, a) the
 *                         padded vertical convolution with the Green's kernel
 *                         of the plan's internal table (the time of the last
 *                         GREEN_FILL or solve), scaled by 4πG/(nx·ny·2nz).
 *                         For SBP_F32 the (0,0) column is left to the FP64
 *                         mean mode and written as zero.
 *   SBP_STAGE_Y_INVERSE : in = out = spectrum; DFT over y with e^{+2πi b y/ny}.
 *   SBP_STAGE_X_INVERSE : in = spectrum, out = real [nz][ny][nx]; the
 *                         half-spectrum inverse x DFT (real part, unscaled).
 *   SBP_STAGE_GREEN_TABLE: in ignored, out = double [ny][nx/2+1][4] holding
 *                         (k², 1 - e^{-kL}, k_p², 1 - e^{-k_p L}) for each
 *                         stored mode and its Hermitian partner at time t:
 *                         the plan's internal table as a solve reads it,
 *                         computed in FP64 and stored in the plan's real type
 *                         (an SBP_F32 plan holds the FP64 values rounded once
 *                         to float), widened to double.
 * The FP32 mean-mode side path is not part of any single stage.
 *
 * The three sweeps of a plan whose solves run them (SBP_OPT_SCHEDULE), on the
 * plan's own workspace in its internal layout (else SBP_ERR_INVALID_ARG):
 *   SBP_STAGE_SWEEP_FORWARD: in = real [nz][ny][nx]; out ignored (may be
 *                         NULL).  Computes the plane sums and leaves the x
 *                         transform and the first y stage (with the second
 *                         stage's twiddles) in the workspace; for most shapes
 *                         it also fills the Green's table for time t.
 *   SBP_STAGE_SWEEP_MIDDLE:  in and out ignored.  The second y stage, the
 *                         padded z pass with the Green's multiply and the
 *                         first inverse y stage, in place, plus the FP64
 *                         mean mode.  Where the forward stage fills no table
 *                         (192- and 256-wide shapes), it evaluates the Green's
 *                         parameters for time t itself.
 *   SBP_STAGE_SWEEP_INVERSE: in ignored; out = real [nz][ny][nx].
 * Run in this order with the same t they give sbp_solve's result bit for
 * bit.
 */
sbp_status sbp_run_stage(sbp_plan p, int stage, const void* in, void* out, double t, void* stream);

/*
 * sbp_solve_noalloc — an FP32 solve that allocates no device memory.
 *
 * The paper has no counterpart: this call exists for host programs that may
 * not allocate device memory while they run (codes that give all device
 * memory to their own pool at start-up, real-time loops that cannot take the
 * device synchronisation an allocation implies, plugin hosts that only hand a
 * library their own buffers).  It computes what sbp_plan_create +
 * sbp_solve(dtype SBP_F32) compute, from the same arguments, with the
 * workspace in one fixed 40 MiB array of device global memory that the
 * library declares statically: every GPU that loads the library holds that
 * array until the process exits.
 *
 * rho, phi: device float arrays [nz][ny][nx], 16-byte aligned, phi == rho
 * allowed, no other overlap.  The sizes, box lengths and parameters follow
 * sbp_plan_create.  A box whose workspace does not fit the 40 MiB (about
 * 256×256×128 cells is the largest cube-like box that does) returns
 * SBP_ERR_SCRATCH_LIMIT before touching the device.
 *
 * Its tables (twiddles, k_z², the FP64 k = 0 kernel) are built by a kernel
 * inside the array on every call; no host memory is copied.  The first call
 * on each device looks up the array's device address (with that device
 * current) and caches it; make that first call before any CUDA stream
 * capture.  Every call on a device shares the array, which keeps the
 * last call's contents (every byte a call reads is written earlier in the
 * same call, so nothing needs clearing).  Calls whose work overlaps on the
 * GPU, for example on two streams, race on the array: order them.
 */
sbp_status sbp_solve_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz,
                             double q, double Omega, double G,
                             const float* rho, float* phi, double t, void* stream);

/* sbp_batch_info — what one sbp_solve_batched call over exactly these
 * (plans, rho, phi) launches, once its graph exists (after the first call):
 * *launches = kernels per call, *grouped_boxes = boxes solved by grouped
 * three-sweep launches (one launch per sweep for all boxes of a shape).
 * Either output may be NULL.  SBP_ERR_INVALID_ARG if no graph is cached for
 * the tuple.  Not part of the paper's method: a report of the schedule. */
sbp_status sbp_batch_info(int nbox, const sbp_plan* plans, const void* const* rho, void* const* phi,
                          int* launches, int* grouped_boxes);

/* sbp_batch_run_stage — one sweep of one group of a cached batch, alone (for
 * stage-level tests and for timing a grouped launch as the batch runs it).
 * The tuple (plans, rho, phi) must have a graph from an earlier
 * sbp_solve_batched call; (nx, ny, nz) picks the group of boxes of that
 * shape that runs grouped sweeps; stage is SBP_STAGE_SWEEP_FORWARD, _MIDDLE
 * or _INVERSE.  The launch covers every box of the group with the shear
 * times of the last sbp_solve_batched call, reading and writing the plans'
 * workspaces and the tuple's rho (forward) or phi (inverse) like the graph
 * does.  Run in order, the three stages give the batched result of those
 * boxes.  SBP_ERR_INVALID_ARG if no such graph or group.  Not part of the
 * paper's method. */
sbp_status sbp_batch_run_stage(int nbox, const sbp_plan* plans, const void* const* rho, void* const* phi,
                               int nx, int ny, int nz, int stage, void* stream);

/* sbp_plan_query — what a plan's solves do now (not part of the paper's
 * method; for callers that report or schedule work).  what:
 *   SBP_QUERY_SCHEDULE (1): 1 = five passes, 2 = three sweeps (see
 *       SBP_OPT_SCHEDULE), after the automatic choice;
 *   SBP_QUERY_LAUNCHES_PER_SOLVE (2): kernels one sbp_solve launches.
 * *value receives the answer.  NULL plan or value, or an unknown `what`:
 * SBP_ERR_INVALID_ARG. */
enum { SBP_QUERY_SCHEDULE = 1, SBP_QUERY_LAUNCHES_PER_SOLVE = 2 };
sbp_status sbp_plan_query(sbp_plan p, int what, double* value);

/* sbp_version — library version string. */
const char* sbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SBP_H */
