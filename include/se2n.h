/*
 * se2n.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of SE(2,N) hypoelliptic-diffusion inpainting (Boscain, Chertovskih,
 * Gauthier, Remizov, "Hypoelliptic diffusion and human vision: a
 * semi-discrete new twist").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units. The diffusion is written in pixel units,
 *     dpsi_r/dt = -a_r^2 psi_r + beta (psi_{r+1} - 2 psi_r + psi_{r-1}),
 *     a_r = wx cos(th_r) + wy sin(th_r),  wx = sin(2 pi l/W), wy = sin(2 pi k/H),
 * for the DFT coefficient (k,l) of every angle plane. This is eq. (4.2)
 * of the paper (Theorem 2) with unit mesh step; se2n_params_from_paper maps
 * the paper's (alpha, T) on an M x M image to (beta, T) here exactly.
 * Angles: th_r = pi r / N (directions, the paper's projectivised picture),
 * or 2 pi r / N when the plan is created with angle_conv = 1.
 *
 * Layout. Images are row-major [H][W] (x = column, y = row); the lifted
 * volume is row-major [N][H][W] of interleaved complex float (8 bytes per
 * element, real then imaginary). Masks and bin maps are [H][W] uint8.
 *
 * Memory. Every pointer argument is DEVICE memory owned by the caller,
 * except in se2n_inpaint_host. The plan owns only its cuFFT plans and small
 * work buffers. Volumes must be 16-byte aligned, images 8-byte aligned, masks
 * and bin maps 2-byte aligned (any cudaMalloc / torch allocation is).
 *
 * Streams and devices. Work is enqueued on the plan's stream (set at
 * creation or by se2n_plan_set_stream) and every call returns after
 * enqueueing, except se2n_inpaint_host which returns when the result is in
 * host memory. Calls must be made with the plan's device current.
 *
 * Errors. Every call returns an se2n_status; nothing is thrown and no device
 * code traps. Arguments are validated on the host before anything is
 * enqueued; on SE2N_EINVAL nothing was enqueued. A CUDA or cuFFT failure
 * returns SE2N_ECUDA / SE2N_ECUFFT and the CUDA error is kept for
 * se2n_plan_last_cuda_error.
 */
#ifndef SE2N_H
#define SE2N_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SE2N_API __attribute__((visibility("default")))
#else
#define SE2N_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum se2n_status {
    SE2N_OK = 0,
    SE2N_EINVAL = 1,        /* bad argument: null/host/misaligned pointer, size, parameter */
    SE2N_ENOMEM = 2,        /* a device or host allocation failed */
    SE2N_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SE2N_ECUFFT = 4,        /* a cuFFT call failed */
    SE2N_EUNSUPPORTED = 5,  /* valid request the library has no kernel for (e.g. an N without an instantiation) */
    SE2N_ENUMERIC = 6       /* parameters outside the range the FP32 scheme resolves */
} se2n_status;

/* Value of a bin-map entry for a "flat" pixel, lifted to every angle. */
#define SE2N_BIN_FLAT 255

/* Projection modes (Section 1.2.4 of the paper: maximum or average). */
#define SE2N_PROJ_MAX 0
#define SE2N_PROJ_MEAN 1

/* se2n_diffuse flags. */
#define SE2N_DIFFUSE_SM_FP64 1     /* Sherman-Morrison correction scalars in FP64 */
#define SE2N_DIFFUSE_SPLIT_DIAG 2  /* keep a_r^2/beta apart from the angular second difference
                                      (always on when beta * T > 8, see se2n_diffuse) */
#define SE2N_DIFFUSE_FULL_CORRECTION 4  /* apply the corner correction on every angle (no truncation) */
/* Integrate by the S-step propagator: for every class of frequencies that
 * share it (rows s, H/2 - s as they are and rows H/2 + s, H - s with the
 * angles reversed, times columns l and (W/2 - l) mod W) the matrix
 * (B-^{-1} B+)^S - I is built once in FP32 by the powering program of
 * se2n_prop_chain, in increment form, and applied as one N x N product per frequency (Section 4: the
 * integration over an interval is one linear map). The same result as S
 * Crank-Nicolson steps up to rounding. The plan keeps the matrices
 * (symmetric; by cyclic diagonals, 4 N (N/2 + 1) bytes a class, or as rows,
 * 4 N^2 bytes a class, for the column pass below and for N = 64 on the
 * Hermitian half, where they are applied 16 classes of one row slot at a
 * time: about H W N^2 / 4 bytes in all) and reuses them while beta dt, S,
 * the spectrum half and the storage
 * stay the same, so the intervals of one inpaint build them once. N = 16,
 * 30, 32 or 64 (else SE2N_EUNSUPPORTED); N = 30 is built and stored as
 * 32 x 32 matrices whose last two rows and columns are zero (the bytes of
 * N = 32). The other flags do not apply.
 * In se2n_inpaint on the Hermitian half with N = 16, 30 or 32 and H, W each one
 * of 64, 128, 256, 384, 512, 768, 1024, this flag alone selects the row and column passes: the
 * volume stays row-transformed between intervals in a plan buffer of
 * 8 (W/2 + 1) H N bytes, each interval is one kernel a column (DFT along y,
 * propagators, inverse DFT) and one kernel a row (real DFTs along x around
 * the restoration), and no cuFFT call is made. The first such call
 * allocates that buffer and a second stream of the plan, on which each
 * build runs beside the orientation and the lift (ordered after the work
 * already on the plan's stream, joined before the first column pass);
 * call once before capturing se2n_inpaint into a graph.
 * Accuracy guard: the FP32 powering in increment form cancels digits when
 * a Crank-Nicolson factor (1 - dt lambda/2) / (1 + dt lambda/2) of the
 * system approaches -1 (stiff modes at large beta dt). The flag is therefore
 * honoured only where every such factor is >= 0, i.e. dt (2 + 4 beta) <= 2
 * (lambda <= max a_r^2 + 4 beta <= 2 + 4 beta); for a larger dt the call runs
 * the step-by-step kernel instead (same result within the 1e-5 bound; the
 * plan's profile then counts no propagator build). */
#define SE2N_DIFFUSE_PROPAGATOR 8

/* Largest N the library has kernels for. */
#define SE2N_MAX_N 64

/* Longest powering program of se2n_prop_chain. */
#define SE2N_PROP_CHAIN_MAX 64

typedef struct se2n_plan se2n_plan;

/* Parameters of the whole method (pixel units).
 *   T        total diffusion time; each of `rounds` restoration intervals
 *            integrates T/rounds in `steps` Crank-Nicolson steps.
 *   rounds   the paper's n (number of static-restoration treatments).
 *   eps      the paper's epsilon in sigma = (eps h(0) + (1-eps) h(t_i)) / h(t_i).
 *   sigma_smooth  Gaussian smoothing of the lift, in pixels.
 *   flat_tol a pixel whose smoothed gradient is <= flat_tol * max|grad| is
 *            lifted to every angle.
 *   proj     SE2N_PROJ_MAX or SE2N_PROJ_MEAN.
 *   final_mix  1: restore once more after the last interval (not in the paper).
 *   guard    restoration divides by h(t_i) only where h(t_i) > guard * h(0)
 *            (relative; 0.1 keeps sigma <= 5.5 at eps = 0.5).
 *   diffuse_flags  SE2N_DIFFUSE_* flags passed to every diffusion.
 *   reinject 1: the result is the inpainted image, f on the known pixels
 *            (mask != 0) and the projection only on the corrupted ones;
 *            0: the projection everywhere (default).
 *   full_spectrum  0 (default): the lifted volume is real, so its spectrum
 *            is Hermitian and the system of frequency (-k, -l) is that of
 *            (k, l) conjugated (a_r^2 is even in the frequency; Theorem 2):
 *            se2n_inpaint integrates the H (W/2 + 1) frequencies l <= W/2
 *            with real-to-complex transforms. 1: all H W frequencies with
 *            complex transforms. Same result up to rounding. The volume
 *            argument of se2n_inpaint is [N][H][W] complex in both cases.
 *   dynamic  1: dynamic restoration (Section 5.3): before every restoration
 *            the good set grows by one step of se2n_dr_grow (starting from
 *            the known pixels), and the restoration pulls every good pixel to
 *            its reference (f for a known pixel, its value when it joined for
 *            the others); reinject still keeps f on the known pixels only.
 *            0: static restoration on the known pixels (default). */
typedef struct se2n_params {
    int N;
    double beta;
    double T;
    int steps;
    int rounds;
    double eps;
    double sigma_smooth;
    double flat_tol;
    int proj;
    int final_mix;
    double guard;
    int diffuse_flags;
    int reinject;
    int full_spectrum;
    int dynamic;
} se2n_params;

/* Fill p with the defaults: N=32, beta=0.25, T=2, steps=100, rounds=1,
 * eps=0.5, sigma_smooth=1, flat_tol=1e-4, proj=max, final_mix=0,
 * guard=0.1, diffuse_flags=0, reinject=0, full_spectrum=0, dynamic=0.
 * SE2N_EINVAL if p is NULL. */
SE2N_API se2n_status se2n_params_default(se2n_params *p);

/* Map the paper's weighting alpha and time T_paper on an M x M image with N
 * angles to pixel units. eq. (2.14): beta_N = alpha (N / 2 pi)^2;
 * eq. (4.1) has mesh step 1/sqrt(M) and a factor 1/2, hence
 * beta = beta_N / M and T = (M/2) T_paper. SE2N_EINVAL for null outputs,
 * M < 2, N < 3, alpha < 0 or T_paper < 0. */
SE2N_API se2n_status se2n_params_from_paper(double alpha, double T_paper, int M, int N,
                                   double *beta_out, double *T_out);

/* Human-readable name of a status (static storage, never NULL). */
SE2N_API const char *se2n_status_string(se2n_status s);

/* The program by which the propagator build (SE2N_DIFFUSE_PROPAGATOR) raises
 * the one-step matrix M to the power S = steps; host only, for inspection.
 * It works on two matrices in increment form, D_m = M^m - I: P, which starts
 * as D_1, and R, which starts empty. Op 0 squares P (D_p -> D_2p: 2 P + P P
 * into P); op 1 squares R into P (D_r -> D_2r); op 2 combines
 * (D_r, D_p -> D_r+p: R + P + R P into R); op 3 copies P into R. Every op but
 * the copy is one N x N product. For S <= 4096 the program has the fewest
 * products of all such two-matrix programs (then the fewest copies), found
 * by a search; above, it is binary powering (lowest bit first). Writes the
 * ops to ops[0 .. *len - 1] and *in_r = 1 when the result ends in R, 0 in P.
 * SE2N_EINVAL for steps < 1, null pointers or cap < the program's length
 * (SE2N_PROP_CHAIN_MAX always suffices). */
SE2N_API se2n_status se2n_prop_chain(int steps, unsigned char *ops, int cap, int *len, int *in_r);

/* Create a plan for H x W images with N angles. H and W even (>= 2), N one
 * of 4, 8, 12, 16, 24, 30, 32, 48, 64 (else SE2N_EUNSUPPORTED), angle_conv 0
 * (th_r = pi r/N) or 1 (2 pi r/N). stream is a cudaStream_t (NULL = the
 * legacy default stream). Allocates the cuFFT plans (batch N over the
 * volume, batch 1 and 2 over one plane) and a work area of about 24 H W
 * bytes. *out is set only on SE2N_OK. */
SE2N_API se2n_status se2n_plan_create(se2n_plan **out, int H, int W, int N, int angle_conv, void *stream);

/* Release everything the plan owns (after synchronizing its stream). NULL is a no-op. */
SE2N_API se2n_status se2n_plan_destroy(se2n_plan *plan);

/* Change the stream later calls enqueue on. */
SE2N_API se2n_status se2n_plan_set_stream(se2n_plan *plan, void *stream);

/* Last CUDA error code (a cudaError_t value) seen by the plan, 0 if none. */
SE2N_API int se2n_plan_last_cuda_error(const se2n_plan *plan);

/* Direction bin of every pixel (Section 1.2.4, first item: smooth with a
 * Gaussian, take the gradient, both in the FFT domain, lift to the closest
 * angle). f0 = f * (mask != 0) is smoothed by exp(-2 pi^2 sigma^2 ((k/H)^2 +
 * (l/W)^2)) and differentiated by i 2 pi l/W, i 2 pi k/H (signed
 * frequencies, Nyquist term 0); the level-line direction phi = atan2(gy,gx) +
 * pi/2 (mod pi) goes to bin floor(phi / dth + 1/2) mod N, dth = pi/N (or
 * 2 pi/N). A pixel with |grad| <= flat_tol max|grad| gets SE2N_BIN_FLAT.
 * f [H][W] float, mask [H][W] uint8 (nonzero = known), bins [H][W] uint8 out.
 * sigma > 0, flat_tol >= 0. Decided in FP32: at pixels whose angle lies
 * within FP32 rounding of a bin boundary, or whose |grad| lies within FP32
 * rounding of the flat threshold, either neighbouring choice may come out. */
SE2N_API se2n_status se2n_orient(se2n_plan *plan, const float *f, const uint8_t *mask, double sigma,
                        double flat_tol, uint8_t *bins);

/* Lift (Section 1.2.4): vol[r][y][x] = f0(x,y) if r is the pixel's bin (every
 * r if the bin is SE2N_BIN_FLAT), else 0; imaginary parts 0. bins values must
 * be < N or SE2N_BIN_FLAT (other values lift to no angle). vol is written
 * completely (8 N H W bytes). */
SE2N_API se2n_status se2n_lift(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins,
                      void *vol);

/* Unnormalised 2-D DFT of every angle plane, in place (Theorem 2): cuFFT C2C. */
SE2N_API se2n_status se2n_forward(se2n_plan *plan, void *vol);

/* Inverse 2-D DFT of every angle plane including 1/(H W), in place. */
SE2N_API se2n_status se2n_inverse(se2n_plan *plan, void *vol);

/* Crank-Nicolson integration of eq. (4.2) for every frequency of the
 * transformed volume, in place: steps steps of dt = T/steps,
 *     (I - dt/2 A) psi_new = (I + dt/2 A) psi,  A = -diag(a_r^2) + beta L,
 * L the cyclic second difference (Section 4, remark after Theorem 2: CN, a
 * tridiagonal matrix with two corner entries). All steps of a frequency run
 * in one launch with the N-vector in registers; HBM is read and written
 * once. beta > 0 (the jump rate of Section 2), T >= 0 (T = 0 is a no-op),
 * steps >= 1, beta*dt >= 1e-30 and beta*dt <= 1e3 (else SE2N_ENUMERIC).
 * flags: SE2N_DIFFUSE_SM_FP64 computes the corner (Sherman-Morrison)
 * correction scalars in FP64. SE2N_DIFFUSE_SPLIT_DIAG forms the right-hand
 * side as (psi_{r-1} + psi_{r+1} - 2 psi_r) - (a_r^2/beta) psi_r instead of
 * with the fused coefficient 2 + a_r^2/beta, whose FP32 rounding perturbs
 * decay rates by ~1.2e-7 beta per unit time; it costs one FMA more per angle
 * and is selected automatically when beta * T > 8.
 * When beta*dt <= ~0.067 (no FP64 flag), a packed fast path runs: the corner
 * correction vector decays by a factor <= 1e-9 within 6 angles of the tear,
 * so it is applied on those angles only (below FP32 resolution elsewhere);
 * SE2N_DIFFUSE_FULL_CORRECTION forces the general kernel. */
SE2N_API se2n_status se2n_diffuse(se2n_plan *plan, void *vol_hat, double beta, double T, int steps, int flags);

/* The same integration for a row shard of the full spectrum: vol_rows holds
 * rows k0 .. k0 + rows - 1 of every angle plane, [N][rows][W] complex,
 * contiguous (the frequencies one GPU owns when a single image is spread
 * over several GPUs: Theorem 2 makes every frequency's system independent,
 * so any set of frequencies can be integrated apart from the rest). The
 * plan's H, W, N and angle grid fix the coefficients a_r of row k0 + i.
 * 0 <= k0, rows >= 1, k0 + rows <= H, else SE2N_EINVAL; flags as for
 * se2n_diffuse except SE2N_DIFFUSE_PROPAGATOR (SE2N_EUNSUPPORTED). */
SE2N_API se2n_status se2n_diffuse_rows(se2n_plan *plan, void *vol_rows, int k0, int rows, double beta, double T,
                                       int steps, int flags);

/* One step of dynamic restoration (Section 5.3) on the real part of the
 * (normalised) complex volume vol [N][H][W]: with h = max_r Re vol_r, a pixel
 * that is bad in mask_in (0) and has a good 8-neighbour becomes good when h
 * exceeds the mean of h over the bad pixels of its 3x3 block inside the image
 * (the pixel included; summed in FP32 row by row, then one division). Every
 * decision uses mask_in. mask_out [H][W] receives the new set (1 good, 0 bad)
 * and must not overlap mask_in; fref [H][W] floats and bins [H][W] bytes, the
 * reference value and orientation bin the restoration pulls a good pixel to,
 * are set for the pixels that join (fref = h, bins = the first angle with the
 * largest value) and left alone elsewhere. Device memory, enqueued on the
 * plan's stream; the plan allocates 12 H W bytes of state on first use.
 * se2n_inpaint does this before every restoration when params.dynamic = 1. */
SE2N_API se2n_status se2n_dr_grow(se2n_plan *plan, const void *vol, const uint8_t *mask_in, uint8_t *mask_out,
                                  float *fref, uint8_t *bins);

/* Static restoration (Section 5, SR) on the real volume, in place: with
 * h(t) = max_r Re vol_r and h(0) = max_r of the lift of (f, mask, bins), a
 * known pixel (mask != 0) with h(t) > guard h(0) has every angle scaled by
 * sigma = (eps h(0) + (1-eps) h(t)) / h(t); a known pixel with
 * h(t) <= guard h(0) (or h(t) <= 0) becomes eps * lift + (1-eps) * Re vol,
 * which moves its maximum to about the same value without dividing by a
 * near-zero h(t). Imaginary parts are set to 0
 * everywhere. 0 <= eps <= 1. */
SE2N_API se2n_status se2n_mix(se2n_plan *plan, void *vol, const float *f, const uint8_t *mask,
                     const uint8_t *bins, double eps, double guard);

/* Static restoration (Section 5, SR) with h(t) given: h_t [H][W] float is
 * the maximum over ALL N angles of the real volume at the restoration time,
 * of which vol may hold only a subset of the planes (an angle shard: a plan
 * created with that many planes, and bins renumbered so that a pixel lifted
 * to an angle outside the shard names no plane of it, 0 .. 254, or stays
 * SE2N_BIN_FLAT). h(0) comes from f itself (the lift's maximum over all
 * angles: f, or max(f, 0) for a pixel on one angle). The rule and the guard
 * are se2n_mix's. */
SE2N_API se2n_status se2n_mix_given(se2n_plan *plan, void *vol, const float *f, const uint8_t *mask,
                                    const uint8_t *bins, const float *h_t, double eps, double guard);

/* Projection to the image (Section 1.2.4): out = max_r Re vol_r
 * (SE2N_PROJ_MAX) or the mean over r (SE2N_PROJ_MEAN). out [H][W] float. */
SE2N_API se2n_status se2n_project(se2n_plan *plan, const void *vol, int proj, float *out);

/* The whole method (Section 5, static restoration): bins (from se2n_orient
 * with p->sigma_smooth and p->flat_tol, or the caller's bins_in if not NULL),
 * lift, forward DFT, then p->rounds intervals of T/rounds: the first from
 * the lift, each later one from the restored state (the restoration at t_0
 * is the identity); the state at T is inverted, optionally restored once
 * more (final_mix), and projected to out. vol [N][H][W] complex is caller
 * scratch, overwritten; out [H][W] float. p->N must equal the plan's N. */
SE2N_API se2n_status se2n_inpaint(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins_in,
                         const se2n_params *p, void *vol, float *out);

/* se2n_inpaint from HOST buffers: copies f and mask to the device, runs the
 * method on plan-owned device buffers (allocated on the first call: the
 * volume, 8 N H W bytes, plus the images) and copies the projected image
 * back to out_host. Returns when out_host holds the result. f_host, mask_host
 * and out_host are host memory (pinned memory makes the copies faster). */
SE2N_API se2n_status se2n_inpaint_host(se2n_plan *plan, const float *f_host, const uint8_t *mask_host,
                              const se2n_params *p, float *out_host);

/* Forget the S-step propagators the plan keeps for SE2N_DIFFUSE_PROPAGATOR:
 * the next such call builds them again. free_memory != 0 also releases their
 * device memory (allocated again on next use). Enqueues nothing; waits for
 * the plan's stream (and a build still running on its second stream) first
 * when it frees. */
SE2N_API se2n_status se2n_plan_drop_propagators(se2n_plan *plan, int free_memory);

/* Tuning of the diffusion launch (used by the autotuner): threads per
 * frequency P (1, 2 or 4; 0 = default for the plan's N), threads per block
 * (multiple of 32, <= 384; the packed FP32 kernels take up to 256 below
 * N = 48 and 384 from N = 48 on, the others 256, and a larger value is
 * lowered to that) and blocks (0 = as many as fit on the device at once).
 * block_threads = 0 restores the default shape, which ignores blocks: 128
 * threads a block and one frequency group a thread for the packed kernels
 * below N = 48, one resident 384-thread block an SM for them from N = 48 on,
 * and 256-thread resident blocks for the others. SE2N_EUNSUPPORTED if no
 * kernel exists for (N, P). */
SE2N_API se2n_status se2n_plan_tune_diffuse(se2n_plan *plan, int threads_per_freq, int block_threads, int blocks);

/* Resource use of the current diffusion kernel choice: registers per thread,
 * resident blocks per SM and threads per frequency. Any output may be NULL. */
SE2N_API se2n_status se2n_plan_diffuse_info(se2n_plan *plan, int *regs_per_thread, int *blocks_per_sm,
                                   int *threads_per_freq);

/* Stage timing. When enabled, the plan brackets every stage it enqueues
 * with CUDA events on its stream and counts its own kernel launches (cuFFT's
 * kernels are not counted as launches of this library). Stages: */
#define SE2N_STAGE_ORIENT 0
#define SE2N_STAGE_LIFT 1
#define SE2N_STAGE_FFT 2      /* forward and inverse DFTs (cuFFT) */
#define SE2N_STAGE_DIFFUSE 3
#define SE2N_STAGE_MIX 4
#define SE2N_STAGE_PROJECT 5
#define SE2N_STAGE_DR 6       /* growth steps of dynamic restoration */
#define SE2N_STAGE_PROPAGATOR 7  /* building S-step propagators (applying them counts as diffusion) */
#define SE2N_NUM_STAGES 8

typedef struct se2n_profile {
    double ms[SE2N_NUM_STAGES];       /* device time accumulated per stage, milliseconds */
    long long calls[SE2N_NUM_STAGES]; /* stage executions timed */
    long long kernels;                /* kernels of this library launched (counted even when timing is off) */
} se2n_profile;

/* Turn stage timing on (1) or off (0); either way the accumulators are reset. */
SE2N_API se2n_status se2n_plan_profile(se2n_plan *plan, int enable);

/* Read the accumulated timings (synchronizes the plan's stream first);
 * reset != 0 clears them afterwards. */
SE2N_API se2n_status se2n_plan_profile_read(se2n_plan *plan, se2n_profile *out, int reset);

/* ---------------------------------------------------------------------------
 * Batches: many images of uneven size and N through one persistent,
 * graph-captured diffusion launch per restoration interval.
 *
 * se2n_batch_create plans the whole batch once: a cuFFT plan per distinct
 * (H, W, N), device storage for every lifted volume and bin map, the work
 * items of the persistent diffusion kernel, and a CUDA graph of the complete
 * method (orientation, lift, DFT, diffusion, restoration, inverse DFT,
 * projection) for every image, captured on the batch's stream. Each warp of
 * the persistent kernel claims (image, frequency-tile) items from an atomic
 * counter; the tile size, block size and threads per frequency are taken
 * from the built-in table or, with SE2N_BATCH_AUTOTUNE, chosen by timing
 * the candidates on this batch. se2n_batch_run replays the graph.
 * ------------------------------------------------------------------------- */

typedef struct se2n_image_desc {
    const float *f;       /* [H][W] device image */
    const uint8_t *mask;  /* [H][W] device mask, nonzero = known */
    float *out;           /* [H][W] device output image */
    const uint8_t *bins;  /* [H][W] device bin map to use, or NULL to compute it (se2n_orient) */
    int H, W, N;          /* H, W even; N one of 16, 32, 64 */
} se2n_image_desc;

typedef struct se2n_batch se2n_batch;

#define SE2N_BATCH_AUTOTUNE 1

typedef struct se2n_batch_info {
    int images;
    int items;              /* work items of the persistent kernel */
    int tile_passes;        /* warp passes (32/P frequencies each) per item */
    int block, blocks;      /* launch shape of the persistent kernel */
    int p16, p32, p64;      /* threads per frequency for N = 16, 32, 64 */
    int fast, split;        /* packed fast path; split diagonal */
    int candidates;         /* launch shapes timed by the autotuner (0 if not run) */
    double best_ms, worst_ms;        /* their fastest and slowest diffusion time */
    double updates_per_run;          /* sum of H W N steps rounds over the images */
    double volume_bytes;             /* device bytes of the lifted volumes */
    int prop_images;                 /* images integrated by their shape's propagators */
    double step_updates;             /* frequencies x N x steps of one interval the persistent kernel integrates */
    int fused_images;                /* of prop_images, those whose whole inpaint runs on the row and column passes */
} se2n_batch_info;

/* Build a batch of `count` images. p->N is ignored (each image has its
 * own); every other field of p applies to all images. angle_conv as in
 * se2n_plan_create. flags: SE2N_BATCH_AUTOTUNE. The image, mask and output
 * buffers must stay valid while the batch is used. Allocates about
 * 8 N H W + H W bytes per image plus the plans. Synchronizes the stream.
 * A NULL (legacy default) stream is replaced by a blocking stream the batch
 * creates, since graphs cannot be captured on the legacy stream; it is
 * ordered with the caller's legacy-stream work. With SE2N_DIFFUSE_PROPAGATOR
 * in p->diffuse_flags, the images of each distinct (H, W, N) are integrated
 * by that shape's S-step propagators (built once a run, shared by the images)
 * when that is estimated to cost less than stepping them, the others by the
 * persistent step-by-step kernel; se2n_batch_get_info reports how many.
 * When every image takes propagators (on the Hermitian half), the graph runs
 * the shapes side by side: each shape's images in turn, as se2n_inpaint
 * runs one image, on a branch of their own. */
SE2N_API se2n_status se2n_batch_create(se2n_batch **out, const se2n_image_desc *imgs, int count,
                                       const se2n_params *p, int angle_conv, int flags, void *stream);

/* Run the whole method for every image of the batch (one graph launch). */
SE2N_API se2n_status se2n_batch_run(se2n_batch *b);

/* The same results computed the plain way: se2n_inpaint on each image in
 * turn (one diffusion launch per image and interval; images that take
 * propagators use the separate apply, and each shape's propagators are
 * built again, as in se2n_batch_run). Bitwise equal to se2n_batch_run; kept
 * as the comparison baseline. */
SE2N_API se2n_status se2n_batch_run_per_image(se2n_batch *b);

/* One persistent diffusion launch over the batch's volumes as they stand
 * (one interval of T/rounds in `steps` steps), outside the graph: for timing
 * the kernel on its own. */
SE2N_API se2n_status se2n_batch_run_diffusion(se2n_batch *b);

SE2N_API se2n_status se2n_batch_get_info(se2n_batch *b, se2n_batch_info *out);

/* Release everything (after synchronizing the stream). NULL is a no-op. */
SE2N_API se2n_status se2n_batch_destroy(se2n_batch *b);

/* ---------------------------------------------------------------------------
 * Learned surrogate (not in the paper): a 4-level U-Net with 32-64-128-256
 * channels, BF16 weights and activations with FP32 accumulation, trained by
 * this library's own forward and backward kernels on (corrupted image,
 * method output) pairs generated by se2n_inpaint / se2n_batch_run. The
 * output is the masked input plus the network's correction,
 *     out = f (mask != 0) + head(decoder),
 * so the network learns only what the method changes. The method stays the
 * judge: se2n_surrogate_inpaint falls back to it for every image whose
 * output misses its own known pixels by more than a threshold (RMS over the
 * known pixels).
 *
 * Layout: images are [count][H][W] float32 and uint8 masks on the device,
 * H and W multiples of 8. Parameters form one flat FP32 vector: for each of
 * the 14 3x3 conv layers (enc0a 8->32, enc0b 32->32, enc1a 32->64, enc1b,
 * enc2a 64->128, enc2b, enc3a 128->256, enc3b, dec2a 384->128, dec2b,
 * dec1a 192->64, dec1b, dec0a 96->32, dec0b) W[cout][9][cin] then b[cout],
 * then the 1x1 head w[32], b[1]. All calls run on the stream given at
 * creation.
 * ------------------------------------------------------------------------- */

typedef struct se2n_unet se2n_unet;

/* Allocate a network for up to `batch` images of H x W (weights zero). */
SE2N_API se2n_status se2n_unet_create(se2n_unet **out, int batch, int H, int W, void *stream);
SE2N_API se2n_status se2n_unet_destroy(se2n_unet *u);
SE2N_API se2n_status se2n_unet_param_count(const se2n_unet *u, long long *n);
/* Deterministic initialisation from a seed (resets Adam): He-normal conv
 * weights, zero biases and a zero head, so that the untrained output is the
 * masked input itself. */
SE2N_API se2n_status se2n_unet_init(se2n_unet *u, unsigned long long seed);
/* Host copies of the flat FP32 parameters / gradients (synchronous). Setting
 * the parameters also resets the Adam moments. */
SE2N_API se2n_status se2n_unet_set_params(se2n_unet *u, const float *host);
SE2N_API se2n_status se2n_unet_get_params(se2n_unet *u, float *host);
SE2N_API se2n_status se2n_unet_get_grads(se2n_unet *u, float *host);
/* out [count][H][W] = f (mask != 0) + network(f, mask). */
SE2N_API se2n_status se2n_unet_forward(se2n_unet *u, const float *f, const uint8_t *mask, int count, float *out);
/* Forward, the loss mean((out - target)^2) (written to loss_device if not
 * NULL) and the gradient of every parameter (kept inside for the optimizer,
 * readable with se2n_unet_get_grads). */
SE2N_API se2n_status se2n_unet_backward(se2n_unet *u, const float *f, const uint8_t *mask, const float *target,
                                        int count, float *loss_device);
/* One Adam step with the last gradients (bias-corrected). */
SE2N_API se2n_status se2n_unet_adam(se2n_unet *u, double lr, double beta1, double beta2, double eps);
/* se2n_unet_backward then se2n_unet_adam(lr, 0.9, 0.999, 1e-8). */
SE2N_API se2n_status se2n_unet_train_step(se2n_unet *u, const float *f, const uint8_t *mask, const float *target,
                                          int count, double lr, float *loss_device);
/* Inpaint `count` images with the network; every image whose output differs
 * from f on its known pixels by more than `threshold` (RMS) is redone by the
 * method (se2n_inpaint with plan and p, vol_scratch [N][H][W] complex on the
 * device, enqueued on the plan's stream). residual_host[count] (may be NULL)
 * receives the per-image RMS, *fallbacks the number redone. The plan must be
 * H x W. */
SE2N_API se2n_status se2n_surrogate_inpaint(se2n_unet *u, se2n_plan *plan, const se2n_params *p, const float *f,
                                            const uint8_t *mask, int count, double threshold, void *vol_scratch,
                                            float *out, float *residual_host, int *fallbacks);

/* ---------------------------------------------------------------------------
 * Diffusion that allocates nothing.
 *
 * The paper has no counterpart to this entry point. It exists for callers
 * that cannot let a library call cudaMalloc: applications that own all
 * device memory through their own pool or arena (a framework allocator, an
 * embedded runtime with a fixed memory budget), and latency-critical loops
 * that cannot afford the implicit device-wide synchronisation cudaMalloc and
 * cudaFree may cause.
 *
 * It integrates the same per-frequency Crank-Nicolson systems as
 * se2n_diffuse, with the same per-frequency kernel code, for up to
 * SE2N_NOALLOC_MAX_VOLUMES transformed volumes (N = 16, 32 or 64, H and W
 * even) in one persistent launch, in place. The caller passes the volumes;
 * the only other memory used is a fixed array of SE2N_NOALLOC_SCRATCH_BYTES
 * bytes compiled into the library, which every GPU that loads the library
 * holds until the process exits. No cudaMalloc, cudaFree or allocating
 * library routine is called, and nothing is copied from host memory: the
 * call's records (volume pointers, sizes, angle tables) travel as the launch
 * parameter of a small set-up kernel that writes them into the array and
 * sets its work counter to zero, followed by the diffusion launch. Both are
 * enqueued on `stream` and the call returns without waiting for the GPU.
 *
 * All calls share that array and it keeps the last call's contents; each
 * call rewrites what it needs. Calls that overlap on the GPU (on different
 * streams, or from several threads without ordering) race on the array and
 * give wrong results: order them. The array's device address is looked up
 * on every call (no allocation); the first call on a device also loads the
 * library's device code, so make that first call before any stream capture.
 * flags: SE2N_DIFFUSE_SPLIT_DIAG and SE2N_DIFFUSE_FULL_CORRECTION as for
 * se2n_diffuse (the FP64 correction is not offered here). SE2N_EINVAL for
 * count < 1 or count > SE2N_NOALLOC_MAX_VOLUMES, bad sizes, parameters or
 * pointers; SE2N_EUNSUPPORTED for another N. */
#define SE2N_NOALLOC_MAX_VOLUMES 64
#define SE2N_NOALLOC_SCRATCH_BYTES 8192

typedef struct se2n_volume_desc {
    void *vol_hat;  /* [N][H][W] complex, 16-byte aligned device memory */
    int H, W, N;
} se2n_volume_desc;

SE2N_API se2n_status se2n_diffuse_many_noalloc(const se2n_volume_desc *vols, int count, double beta, double T,
                                               int steps, int angle_conv, int flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SE2N_H */
