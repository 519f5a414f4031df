// Internal declarations shared by the CUDA translation units of libse2n.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <vector>

#include "se2n.h"

struct DrState {
    uint8_t *buf = nullptr;  // one allocation of 12 H W bytes holding the arrays below
    float *fref = nullptr, *h = nullptr;
    uint8_t *mask[2] = {nullptr, nullptr};
    uint8_t *bins = nullptr, *amax = nullptr;
    int cur = 0;  // mask[cur] is the current good set
};

struct se2n_plan {
    int H, W, N, angle_conv;
    long long HW;
    int device;
    cudaStream_t stream;
    cufftHandle fft_vol;   // batch N, [H][W], C2C, in place
    cufftHandle fft_one;   // one plane
    cufftHandle fft_two;   // batch 2 (gradient components)
    // Hermitian-half path (created on first use): the real volume is [N][H][W+2]
    // floats, its spectrum [N][H][Wc] complex in the same memory, Wc = W/2 + 1
    int Wc;
    cufftHandle fft_r2c;   // batch N, R2C, in place
    cufftHandle fft_c2r;   // batch N, C2R, in place
    bool half_ready;
    float2 *spec;          // [3][H][W]: image spectrum, x and y gradient
    unsigned int *gmax;    // one word: max |grad|^2 as float bits
    uint8_t *bins;         // [H][W] bins computed by se2n_inpaint
    // se2n_inpaint_host buffers (allocated on first use)
    float *h_f, *h_out;
    uint8_t *h_mask;
    float2 *h_vol;
    // dynamic restoration state (allocated on first use): the good set
    // (ping-pong), the reference values and bins the restoration pulls the
    // good pixels to, and the image value and argmax angle of the last step
    DrState dr;
    // S-step propagators (SE2N_DIFFUSE_PROPAGATOR), kept for the next call
    // with the same beta dt, S and spectrum half
    float *prop_D;
    size_t prop_bytes;
    bool prop_valid;
    double prop_beta, prop_bdt;
    int prop_steps;
    bool prop_half;
    int prop_fmt;          // storage: PROP_DIAGONALS, PROP_CHUNKS or PROP_ROWS
    // the powering program of S = chain_steps (0: none yet)
    int chain_steps;
    unsigned char chain[SE2N_PROP_CHAIN_MAX];
    int chain_len, chain_in_r;
    // side stream for a build that overlaps the start of an inpaint, and the
    // events that order it after the plan's stream and the plan's stream
    // after it (join_pending until the plan's stream waits on ev_join)
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    bool join_pending;
    // row and column passes of the Hermitian half (se2n_inpaint with
    // propagators): the row-transformed volume [Wc][H][N] complex
    float2 *colbuf;
    float2 *col_tw;        // exp(-2 pi i m / H), m < H
    float2 *row_tw;        // exp(-2 pi i m / W), m < W
    bool col_ready;
    // diffusion launch configuration
    int diffuse_P;         // threads per frequency
    int diffuse_block;     // threads per block; 0 = the default shape for N
    int diffuse_blocks;    // 0 = fill the device
    int num_sms;
    int last_cuda_error;
    // stage timing (se2n_plan_profile): event pairs per stage, reused
    bool profiling;
    std::vector<cudaEvent_t> stage_ev[SE2N_NUM_STAGES];
    int stage_used[SE2N_NUM_STAGES];
    double prof_ms[SE2N_NUM_STAGES];
    long long prof_calls[SE2N_NUM_STAGES];
    long long kernels;  // own kernel launches
};

// Scalars of one diffusion call, shared by every frequency.
struct StepParams {
    int steps;
    float inv_c;      // 2 / (beta dt): the left CN matrix divided by beta dt / 2
    float inv_beta;
    double inv_c_d;   // the same in FP64 (Sherman-Morrison scalars in FP64)
    double inv_beta_d;
};

// Parameters of one single-image diffusion launch (kernel parameter space:
// read through the constant bank, so the angle tables cost no loads).
struct DiffuseArgs {
    float2 *vol;
    long long HW;  // frequencies per plane (the plane's stride in complex elements)
    int H, W;
    int Wc;        // stored columns per row: W, or W/2 + 1 for the Hermitian half
    int k0;        // first spectrum row of vol (a row shard), 0 for a whole volume
    StepParams sp;
    float cs[SE2N_MAX_N];
    float sn[SE2N_MAX_N];
};

// Parameters of the propagator kernels (propagator.cu): build D_S for every
// class of frequencies with equal coefficients, or apply it to the volume.
// Ops of the powering program, in increment form D_m = M^m - I:
//   PROP_SQ_P  P <- 2 P + P P  (D_p -> D_2p)
//   PROP_SQ_R  P <- 2 R + R R  (D_r -> D_2r)
//   PROP_ADD   R <- R + P + R P  (D_r, D_p -> D_r+p)
//   PROP_COPY  R <- P
enum PropOp : unsigned char { PROP_SQ_P = 0, PROP_SQ_R = 1, PROP_ADD = 2, PROP_COPY = 3 };

// Storage of the propagators of a plan (PropArgs::rows).
enum : int {
    PROP_DIAGONALS = 0,  // [classes][N/2 + 1][N] cyclic diagonals (the apply of the full spectrum)
    PROP_CHUNKS = 1,     // [classes][N/4][N] float4: row i's entries 4c .. 4c + 3 at float4 c N + i
                         // (the column pass)
    PROP_ROWS = 2        // [classes][N][N] row-major, built classes only (the tiled apply)
};

struct PropArgs {
    float *D;          // D_S = (B-^{-1} B+)^S - I a class, stored as `rows` says
    int rows;          // PROP_DIAGONALS, PROP_CHUNKS or PROP_ROWS
    float2 *vol;       // [N][H][Wc] complex (apply only)
    int H, W, Wc;
    long long HW;      // H * Wc
    int col_slots;     // column classes a row class
    long long classes;
    // classes the build computes: all of them, or with share_t (square
    // planes, Hermitian half) the row slot <= column slot ones, each also
    // stored permuted for its transpose, angle r -> (perm_shift - r) mod N
    // (not with PROP_ROWS: the tiled apply permutes the vectors instead)
    long long items;
    int share_t;
    int perm_shift;
    int steps;         // S
    // the powering program (se2n_prop_chain): ops PROP_* on P (starting as
    // D_1) and R (empty); the result ends in R when chain_in_r
    unsigned char chain[SE2N_PROP_CHAIN_MAX];
    int chain_len;
    int chain_in_r;
    float inv_c;       // 2 / (beta dt)
    float inv_beta;
    int half;          // 1: the Hermitian half (columns l <= W/2), 0: all W columns
    float cs[SE2N_MAX_N];
    float sn[SE2N_MAX_N];
};
bool se2n_prop_supported(int N);  // 16, 30 (stored as 32), 32, 64
int se2n_prop_dim(int N);          // angles of the stored propagator
long long se2n_prop_floats(int N, int fmt = PROP_DIAGONALS);  // stored floats a class
// The storage se2n_launch_prop_apply reads: PROP_ROWS for the tiled apply
// (Hermitian half, N = 64), else PROP_DIAGONALS.
int se2n_prop_apply_fmt(int N, bool half);
int se2n_prop_col_slots(int W, bool half);
long long se2n_prop_classes(int H, int W, bool half);
// Set the kernels' shared-memory attributes for N (before a graph capture).
cudaError_t se2n_prop_prepare(int N);
cudaError_t se2n_launch_prop_build(int N, const PropArgs &a, int num_sms, cudaStream_t s);
cudaError_t se2n_launch_prop_apply(int N, const PropArgs &a, int num_sms, cudaStream_t s);

// colprop.cu: the column pass of one interval on the row-transformed
// Hermitian half [Wc][H][N] (forward DFT along k, x <- x + D_S x with D_S
// stored as rows, inverse DFT along k), one block a column.
struct ColArgs {
    float2 *col;        // [Wc][H][N] complex, in place
    const float *D;     // [classes][N/4][N] float4 (see PropArgs)
    const float2 *tw;   // exp(-2 pi i m / H), m < H
    int H, W, Wc, col_slots;
    int num_sms;        // the device's SMs (the persistent grid's size)
};
bool se2n_col_supported(int N, int H);
cudaError_t se2n_col_prepare(int N, int H);
cudaError_t se2n_launch_col_prop(int N, const ColArgs &a, cudaStream_t s);
// 1 in *host_flag when a column pass gave up waiting for its copy-in (reset clears it)
cudaError_t se2n_col_fault(int *host_flag, bool reset);

// rowfft.cu: the row pass between column passes, one block a row y with all
// its angles: the row-transformed volume [Wc][H][N] is taken back to the
// image (inverse real DFT along x), restored, and transformed again, or the
// row comes from the lift, or goes to the projection or to the real volume.
enum { SE2N_ROW_IN_LIFT = 0, SE2N_ROW_IN_SPEC = 1, SE2N_ROW_IN_REAL = 2 };
enum { SE2N_ROW_OUT_SPEC = 0, SE2N_ROW_OUT_REAL = 1, SE2N_ROW_OUT_PROJ = 2, SE2N_ROW_OUT_H = 3 };
struct RowArgs {
    const float2 *spec_in;  // [Wc][H][N] complex (IN_SPEC)
    float2 *spec_out;       // [Wc][H][N] complex (OUT_SPEC); may be spec_in
    const float *real_in;   // [N][H][W + 2] (IN_REAL)
    float *real_out;        // [N][H][W + 2] (OUT_REAL), unnormalised
    float *proj_out;        // [H][W] (OUT_PROJ)
    const float *f;         // [H][W] image (lift, restoration, reinjection)
    const uint8_t *mask;    // [H][W] known pixels
    const uint8_t *bins;    // [H][W] orientation bins
    const float2 *tw;       // exp(-2 pi i m / W), m < W
    int H, in_mode, out_mode;
    int mix;                // restore after the inverse DFT (IN_SPEC)
    float scale, eps, guard;
    int proj, reinject;     // OUT_PROJ: max or mean over the angles of scale_proj * value
    float scale_proj;
    const float *rf;        // OUT_PROJ: the reinjected image and its known pixels
    const uint8_t *rmask;   //   (f and mask when null)
    float *h_out;           // OUT_H: [H][W] max over the angles of scale * value
    uint8_t *amax_out;      //   and the angle of its first maximum
};
bool se2n_row_supported(int N, int W);
cudaError_t se2n_row_prepare(int N, int W);
cudaError_t se2n_launch_row(int N, int W, const RowArgs &a, cudaStream_t s);

// Host helpers shared by the single-image and batched paths (capi.cu).
StepParams step_params(double beta, double beta_dt, int steps);
// cos/sin of th_r = (pi or 2 pi) r / N for r < count (zero past N), as FP32.
void angle_table(int N, int angle_conv, float *cs, float *sn, int count);

// Launch the diffusion kernel for (N, P, fp64 correction) on `stream`.
// Returns cudaErrorInvalidValue if no instantiation exists.
// `fast` asks for the packed fast path (truncated tear correction); it is
// used when an instantiation exists and sm_fp64 is off.
cudaError_t se2n_launch_diffuse(int N, int P, bool sm_fp64, bool split, bool fast, const DiffuseArgs &a,
                                int block, int blocks, cudaStream_t stream);
// Occupancy query for the same kernel: blocks per SM and registers per thread.
cudaError_t se2n_diffuse_occupancy(int N, int P, bool sm_fp64, bool split, bool fast, int block,
                                   int *blocks_per_sm, int *regs);
// Largest block the chosen kernel accepts (its launch bound).
int se2n_diffuse_block_limit(int N, int P, bool sm_fp64, bool split, bool fast);
// Launch shape of one diffusion launch over `freqs` frequencies: the plan's
// tuned block and grid, or by default 128-thread blocks with one frequency
// group per thread (N < 48, packed kernel) or one resident 384-thread block
// an SM (N >= 48, packed kernel), 256-thread resident blocks otherwise.
cudaError_t se2n_diffuse_shape(int N, int P, bool sm_fp64, bool split, bool fast, int tuned_block,
                               int tuned_blocks, int num_sms, long long freqs, int *block, int *blocks);
// Whether the tear corrections may be truncated for this beta * dt.
bool se2n_diffuse_truncation_ok(double beta_dt);
// Whether an instantiation exists for (N, P).
bool se2n_diffuse_has(int N, int P);
int se2n_diffuse_default_P(int N);

// Pixel kernels (pixel.cu).
cudaError_t se2n_launch_orient_prep(const float *f, const uint8_t *mask, float2 *spec, long long HW,
                                    cudaStream_t s);
cudaError_t se2n_launch_grad_spec(float2 *spec, int H, int W, float sigma, cudaStream_t s);
cudaError_t se2n_launch_grad_max(const float2 *gx, const float2 *gy, long long HW, unsigned int *gmax,
                                 cudaStream_t s);
cudaError_t se2n_launch_bins(const float2 *gx, const float2 *gy, long long HW, const unsigned int *gmax,
                             float flat_tol2, int N, int angle_conv, uint8_t *bins, cudaStream_t s);
cudaError_t se2n_launch_lift(const float *f, const uint8_t *mask, const uint8_t *bins, float2 *vol,
                             long long HW, int N, cudaStream_t s);
cudaError_t se2n_launch_mix(float2 *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                            long long HW, int N, float scale, float eps, float guard, cudaStream_t s);
// The same rule with h(t) given (the maximum over all angles, of which vol
// may hold only some planes); vol already normalised.
cudaError_t se2n_launch_mix_given(float2 *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                                  const float *h_t, long long HW, int N, float eps, float guard, cudaStream_t s);
// out = max_r (or mean_r) of scale * Re vol[r]; where mask != null, pixels
// with mask != 0 take f instead (the inpainted image).
// The same stages on the real volume of the Hermitian-half path: planes of H
// rows of W + 2 floats (in-place R2C layout).
cudaError_t se2n_launch_lift_r(const float *f, const uint8_t *mask, const uint8_t *bins, float *vol, int H, int W,
                               int N, cudaStream_t s);
cudaError_t se2n_launch_mix_r(float *vol, const float *f, const uint8_t *mask, const uint8_t *bins, int H, int W,
                              int N, float scale, float eps, float guard, cudaStream_t s);
cudaError_t se2n_launch_project_r(const float *vol, int H, int W, int N, float scale, int proj, const float *f,
                                  const uint8_t *mask, float *out, cudaStream_t s);
cudaError_t se2n_launch_project(const float2 *vol, long long HW, int N, float scale, int proj, const float *f,
                                const uint8_t *mask, float *out, cudaStream_t s);
cudaError_t se2n_launch_scale(float2 *vol, long long count, float scale, cudaStream_t s);
// Dynamic restoration: h = max_r scale * Re vol[r] and the angle of its first
// maximum (complex [N][HW] volume, or the real half-path layout), then one
// growth step of the good set from mask_in to mask_out (updating fref and bins
// of the pixels that join).
cudaError_t se2n_launch_dr_max(const float2 *vol, long long HW, int N, float scale, float *h, uint8_t *amax,
                               cudaStream_t s);
cudaError_t se2n_launch_dr_max_r(const float *vol, int H, int W, int N, float scale, float *h, uint8_t *amax,
                                 cudaStream_t s);
cudaError_t se2n_launch_dr_grow(const float *h, const uint8_t *amax, const uint8_t *mask_in, uint8_t *mask_out,
                                float *fref, uint8_t *bins, int H, int W, cudaStream_t s);
