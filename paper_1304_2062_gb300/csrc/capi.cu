// C ABI of libse2n: plans, argument validation, cuFFT wiring and the
// orchestration of the whole inpainting method. Every check happens on the
// host before anything is enqueued; device code never traps.
#include <math.h>
#include <new>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "se2n_batch.h"
#include "se2n_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

se2n_status cuda_status(se2n_plan *plan, cudaError_t e) {
    if (e == cudaSuccess) return SE2N_OK;
    if (plan) plan->last_cuda_error = (int)e;
    return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
}

se2n_status cufft_status(cufftResult r) {
    if (r == CUFFT_SUCCESS) return SE2N_OK;
    return r == CUFFT_ALLOC_FAILED ? SE2N_ENOMEM : SE2N_ECUFFT;
}

// Brackets one stage with CUDA events on the plan's stream when timing is on.
struct StageTimer {
    se2n_plan *plan;
    int stage;
    bool on;
    cudaStream_t stream;
    StageTimer(se2n_plan *p, int s, cudaStream_t st = nullptr)
        : plan(p), stage(s), on(p->profiling), stream(st ? st : p->stream) {
        if (!on) return;
        std::vector<cudaEvent_t> &ev = plan->stage_ev[stage];
        const size_t need = 2 * (size_t)plan->stage_used[stage] + 2;
        while (ev.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                (void)cudaGetLastError();
                on = false;
                return;
            }
            ev.push_back(e);
        }
        cudaEventRecord(ev[need - 2], stream);
    }
    ~StageTimer() {
        if (!on) return;
        const int u = plan->stage_used[stage]++;
        cudaEventRecord(plan->stage_ev[stage][2 * u + 1], stream);
    }
};

#define SE2N_TRY(expr)                      \
    do {                                    \
        se2n_status _s = (expr);            \
        if (_s != SE2N_OK) return _s;       \
    } while (0)

// Device (or managed) memory the current device can address; rejects host
// pointers, which a kernel could not use.
bool device_ptr(const void *p, size_t align) {
    if (!p || ((uintptr_t)p % align) != 0) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

se2n_status check_plan(se2n_plan *plan) {
    if (!plan) return SE2N_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return SE2N_EINVAL;
    return SE2N_OK;
}

}  // namespace

StepParams step_params(double beta, double beta_dt, int steps) {
    StepParams sp;
    sp.steps = steps;
    sp.inv_c_d = 2.0 / beta_dt;
    sp.inv_beta_d = 1.0 / beta;
    sp.inv_c = (float)sp.inv_c_d;
    sp.inv_beta = (float)sp.inv_beta_d;
    return sp;
}

void angle_table(int N, int angle_conv, float *cs, float *sn, int count) {
    const double dth = (angle_conv ? 2.0 : 1.0) * kPi / N;
    for (int r = 0; r < count; ++r) {
        cs[r] = r < N ? (float)cos(dth * r) : 0.0f;
        sn[r] = r < N ? (float)sin(dth * r) : 0.0f;
    }
}

namespace {

// Device memory for the plan's propagators (grown when too small, which
// invalidates them).
se2n_status prop_reserve(se2n_plan *plan, bool half, int fmt) {
    const size_t need =
        (size_t)se2n_prop_classes(plan->H, plan->W, half) * (size_t)se2n_prop_floats(plan->N, fmt) * sizeof(float);
    if (plan->prop_bytes >= need) return SE2N_OK;
    cudaFree(plan->prop_D);
    plan->prop_D = nullptr;
    plan->prop_bytes = 0;
    plan->prop_valid = false;
    cudaError_t e = cudaMalloc(&plan->prop_D, need);
    if (e != cudaSuccess) {
        plan->prop_D = nullptr;
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
    }
    plan->prop_bytes = need;
    return SE2N_OK;
}

PropArgs prop_args(se2n_plan *plan, float2 *vol, double beta, double bdt, int steps, bool half, int fmt) {
    PropArgs a{};
    a.vol = vol;
    a.rows = fmt;
    a.H = plan->H;
    a.W = plan->W;
    a.Wc = half ? plan->Wc : plan->W;
    a.HW = (long long)a.H * a.Wc;
    a.half = half ? 1 : 0;
    a.col_slots = se2n_prop_col_slots(plan->W, half);
    a.classes = se2n_prop_classes(plan->H, plan->W, half);
    // square planes on the Hermitian half: a class and its transpose share
    // one build (the angle reflection th -> pi/2 - th maps one operator onto
    // the other; on the 2 pi r / N grid it needs 4 | N)
    a.share_t = half && plan->H == plan->W && (plan->angle_conv == 0 || plan->N % 4 == 0) ? 1 : 0;
    a.perm_shift = plan->angle_conv ? plan->N / 4 : plan->N / 2;
    a.items = a.share_t ? (long long)a.col_slots * (a.col_slots + 1) / 2 : a.classes;
    a.steps = steps;
    a.inv_c = (float)(2.0 / bdt);
    a.inv_beta = (float)(1.0 / beta);
    angle_table(plan->N, plan->angle_conv, a.cs, a.sn, SE2N_MAX_N);
    a.D = plan->prop_D;
    return a;
}

// The plan's side stream and the events that fork work to it and join it back.
se2n_status side_ensure(se2n_plan *plan) {
    if (plan->side) return SE2N_OK;
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        if (st) cudaStreamDestroy(st);
        if (fork) cudaEventDestroy(fork);
        return SE2N_ECUDA;
    }
    plan->side = st;
    plan->ev_fork = fork;
    plan->ev_join = join;
    return SE2N_OK;
}

// The plan's stream waits for the propagators built on the side stream.
void prop_join(se2n_plan *plan) {
    if (!plan->join_pending) return;
    cudaStreamWaitEvent(plan->stream, plan->ev_join, 0);
    plan->join_pending = false;
}

// Whether the propagator form keeps the 1e-5 accuracy of the step kernel.
// The build raises M = B-^-1 B+ to the power S in increment form, D -> 2D + D^2
// for a squaring. For an eigenvalue mu of M that is >= 0, D = mu - 1 lies in
// [-1, 0] and no product cancels; as mu approaches -1 (stiff modes at large
// beta dt), D approaches -2, 2D + D^2 cancels to a small number and FP32
// loses digits at every squaring (measured on the GPU: N = 64, S = 30,
// beta dt = 10 gave 1.3e-5 against the oracle). So propagators are used only
// where every mu = (1 - dt lambda / 2) / (1 + dt lambda / 2) is >= 0, i.e.
// dt lambda <= 2 for the largest eigenvalue lambda of -A; by Gershgorin
// lambda <= max a_r^2 + 4 beta <= 2 + 4 beta (a_r^2 <= wx^2 + wy^2 <= 2).
// Elsewhere the step kernel runs instead.
bool prop_admissible(double beta, double dt) { return dt * (2.0 + 4.0 * beta) <= 2.0; }

// The S-step propagators of every class of frequencies, built when beta dt,
// S, the spectrum half or the storage changed. With side = true the build
// runs on the plan's side stream after everything queued on the plan's
// stream so far (it reads nothing that work writes), overlapping what the
// plan's stream does next until prop_join.
se2n_status prop_ensure(se2n_plan *plan, double beta, double bdt, int steps, bool half, int fmt,
                        bool side = false) {
    if (!se2n_prop_supported(plan->N)) return SE2N_EUNSUPPORTED;
    SE2N_TRY(prop_reserve(plan, half, fmt));
    if (plan->prop_valid && plan->prop_beta == beta && plan->prop_bdt == bdt && plan->prop_steps == steps &&
        plan->prop_half == half && plan->prop_fmt == fmt)
        return SE2N_OK;
    plan->prop_valid = false;
    if (plan->chain_steps != steps) {
        SE2N_TRY(se2n_prop_chain(steps, plan->chain, SE2N_PROP_CHAIN_MAX, &plan->chain_len, &plan->chain_in_r));
        plan->chain_steps = steps;
    }
    PropArgs a = prop_args(plan, nullptr, beta, bdt, steps, half, fmt);
    std::copy(plan->chain, plan->chain + plan->chain_len, a.chain);
    a.chain_len = plan->chain_len;
    a.chain_in_r = plan->chain_in_r;
    cudaStream_t st = plan->stream;
    if (side) {
        SE2N_TRY(side_ensure(plan));
        prop_join(plan);  // an earlier build on the side stream, if any
        if (cudaEventRecord(plan->ev_fork, plan->stream) != cudaSuccess ||
            cudaStreamWaitEvent(plan->side, plan->ev_fork, 0) != cudaSuccess)
            return SE2N_ECUDA;
        st = plan->side;
    }
    {
        StageTimer timer(plan, SE2N_STAGE_PROPAGATOR, st);
        plan->kernels += 1;
        SE2N_TRY(cuda_status(plan, se2n_launch_prop_build(plan->N, a, plan->num_sms, st)));
    }
    if (side) {
        if (cudaEventRecord(plan->ev_join, plan->side) != cudaSuccess) return SE2N_ECUDA;
        plan->join_pending = true;
    }
    plan->prop_valid = true;
    plan->prop_beta = beta;
    plan->prop_bdt = bdt;
    plan->prop_steps = steps;
    plan->prop_half = half;
    plan->prop_fmt = fmt;
    return SE2N_OK;
}

// The propagators applied once to the spectrum vol (by diagonals, or tile
// by tile from rows: se2n_prop_apply_fmt).
se2n_status propagate_impl(se2n_plan *plan, float2 *vol, double beta, double bdt, int steps, bool half) {
    const int fmt = se2n_prop_apply_fmt(plan->N, half);
    SE2N_TRY(prop_ensure(plan, beta, bdt, steps, half, fmt));
    prop_join(plan);
    const PropArgs a = prop_args(plan, vol, beta, bdt, steps, half, fmt);
    StageTimer timer(plan, SE2N_STAGE_DIFFUSE);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_prop_apply(plan->N, a, plan->num_sms, plan->stream));
}

// Row and column passes of the Hermitian half (rowfft.cu, colprop.cu): the
// row-transformed volume [Wc][H][N] complex and the twiddle tables.
bool col_path(const se2n_plan *plan, const se2n_params *p) {
    return !p->full_spectrum && p->diffuse_flags == SE2N_DIFFUSE_PROPAGATOR &&
           prop_admissible(p->beta, p->T / p->rounds / p->steps) && se2n_col_supported(plan->N, plan->H) &&
           se2n_row_supported(plan->N, plan->W);
}

// exp(-2 pi i m / n), m < n, from the exact fraction m / n
se2n_status upload_twiddles(float2 **dst, int n) {
    cudaError_t e = cudaMalloc(dst, (size_t)n * sizeof(float2));
    if (e != cudaSuccess) {
        *dst = nullptr;
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
    }
    std::vector<float2> tw(n);
    for (int m = 0; m < n; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)n;
        tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    }
    return cudaMemcpy(*dst, tw.data(), (size_t)n * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess
               ? SE2N_OK
               : SE2N_ECUDA;
}

se2n_status col_ensure(se2n_plan *plan) {
    if (plan->col_ready) return SE2N_OK;
    if (!plan->colbuf) {
        // N = 30 is held in 32 slots
        cudaError_t e =
            cudaMalloc(&plan->colbuf, (size_t)plan->Wc * se2n_prop_dim(plan->N) * plan->H * sizeof(float2));
        if (e != cudaSuccess) {
            plan->colbuf = nullptr;
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
        }
    }
    if (!plan->col_tw) SE2N_TRY(upload_twiddles(&plan->col_tw, plan->H));
    if (!plan->row_tw) SE2N_TRY(upload_twiddles(&plan->row_tw, plan->W));
    if (cuda_status(plan, se2n_col_prepare(plan->N, plan->H)) != SE2N_OK ||
        cuda_status(plan, se2n_row_prepare(plan->N, plan->W)) != SE2N_OK)
        return SE2N_ECUDA;
    plan->col_ready = true;
    return SE2N_OK;
}

// The row and column passes' buffers, and the propagators: they depend on
// beta dt and S only, so they are built on the side stream while the
// orientation, the lift (and the host copies of se2n_inpaint_host) run.
se2n_status col_start(se2n_plan *plan, const se2n_params *p) {
    SE2N_TRY(col_ensure(plan));
    const double bdt = p->beta * (p->T / p->rounds) / p->steps;
    if (p->T > 0.0 && bdt >= 1e-30 && bdt <= 1e3)
        SE2N_TRY(prop_ensure(plan, p->beta, bdt, p->steps, true, PROP_CHUNKS, true));
    return SE2N_OK;
}

RowArgs row_args(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins, float scale, float eps,
                 float guard) {
    RowArgs r;
    r.spec_in = plan->colbuf;
    r.spec_out = plan->colbuf;
    r.real_in = nullptr;
    r.real_out = nullptr;
    r.proj_out = nullptr;
    r.f = f;
    r.mask = mask;
    r.bins = bins;
    r.tw = plan->row_tw;
    r.H = plan->H;
    r.in_mode = SE2N_ROW_IN_SPEC;
    r.out_mode = SE2N_ROW_OUT_SPEC;
    r.mix = 0;
    r.scale = scale;
    r.eps = eps;
    r.guard = guard;
    r.proj = SE2N_PROJ_MAX;
    r.reinject = 0;
    r.scale_proj = 1.0f;
    r.rf = nullptr;
    r.rmask = nullptr;
    r.h_out = nullptr;
    r.amax_out = nullptr;
    return r;
}

se2n_status row_pass(se2n_plan *plan, const RowArgs &r) {
    StageTimer timer(plan, SE2N_STAGE_FFT);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_row(plan->N, plan->W, r, plan->stream));
}

se2n_status col_diffuse(se2n_plan *plan, double beta, double T, int steps) {
    if (!(beta > 0.0) || !(T >= 0.0) || steps < 1 || !isfinite(beta) || !isfinite(T)) return SE2N_EINVAL;
    if (T == 0.0) return SE2N_OK;
    const double bdt = beta * (T / steps);
    if (!(bdt >= 1e-30 && bdt <= 1e3)) return SE2N_ENUMERIC;
    SE2N_TRY(prop_ensure(plan, beta, bdt, steps, true, PROP_CHUNKS));
    prop_join(plan);
    ColArgs a;
    a.col = plan->colbuf;
    a.D = plan->prop_D;
    a.tw = plan->col_tw;
    a.H = plan->H;
    a.W = plan->W;
    a.Wc = plan->Wc;
    a.col_slots = se2n_prop_col_slots(plan->W, true);
    a.num_sms = plan->num_sms;
    StageTimer timer(plan, SE2N_STAGE_DIFFUSE);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_col_prop(plan->N, a, plan->stream));
}

// half: vol holds the Hermitian half [N][H][W/2 + 1] of the spectrum.
// rows >= 0: vol holds only spectrum rows k0 .. k0 + rows - 1 of every plane
// ([N][rows][W], a row shard of the full spectrum).
se2n_status diffuse_impl(se2n_plan *plan, float2 *vol, double beta, double T, int steps, int flags, bool half = false,
                         int k0 = 0, int rows = -1) {
    if (!(beta > 0.0) || !(T >= 0.0) || steps < 1 || !isfinite(beta) || !isfinite(T)) return SE2N_EINVAL;
    if (flags & ~(SE2N_DIFFUSE_SM_FP64 | SE2N_DIFFUSE_SPLIT_DIAG | SE2N_DIFFUSE_FULL_CORRECTION |
                  SE2N_DIFFUSE_PROPAGATOR))
        return SE2N_EINVAL;
    if (T == 0.0) return SE2N_OK;
    const double dt = T / steps;
    const double bdt = beta * dt;
    if (!(bdt >= 1e-30 && bdt <= 1e3)) return SE2N_ENUMERIC;
    if (flags & SE2N_DIFFUSE_PROPAGATOR) {
        if (!se2n_prop_supported(plan->N) || rows >= 0) return SE2N_EUNSUPPORTED;
        if (prop_admissible(beta, dt)) return propagate_impl(plan, vol, beta, bdt, steps, half);
        flags &= ~SE2N_DIFFUSE_PROPAGATOR;  // stiff: the step kernel keeps the accuracy
    }
    const bool fp64 = (flags & SE2N_DIFFUSE_SM_FP64) != 0;
    // The fused diagonal 2 + a^2/beta perturbs decay rates by ~1.2e-7 beta per
    // unit time; past beta T = 8 that exceeds 1e-6 and the split form is used.
    const bool split = (flags & SE2N_DIFFUSE_SPLIT_DIAG) != 0 || beta * T > 8.0;
    const bool fast = !(flags & SE2N_DIFFUSE_FULL_CORRECTION) && se2n_diffuse_truncation_ok(bdt);

    DiffuseArgs a;
    a.vol = vol;
    a.Wc = half ? plan->Wc : plan->W;
    a.HW = (long long)(rows >= 0 ? rows : plan->H) * a.Wc;
    a.k0 = rows >= 0 ? k0 : 0;
    a.H = plan->H;
    a.W = plan->W;
    a.sp = step_params(beta, bdt, steps);
    angle_table(plan->N, plan->angle_conv, a.cs, a.sn, SE2N_MAX_N);
    const int P = plan->diffuse_P;
    int block = 0, blocks = 0;
    cudaError_t es = se2n_diffuse_shape(plan->N, P, fp64, split, fast, plan->diffuse_block, plan->diffuse_blocks,
                                        plan->num_sms, a.HW, &block, &blocks);
    if (es != cudaSuccess) {
        if (es == cudaErrorInvalidValue && !se2n_diffuse_has(plan->N, P)) return SE2N_EUNSUPPORTED;
        return cuda_status(plan, es);
    }
    StageTimer timer(plan, SE2N_STAGE_DIFFUSE);
    plan->kernels += 1;
    cudaError_t e = se2n_launch_diffuse(plan->N, P, fp64, split, fast, a, block, blocks, plan->stream);
    if (e == cudaErrorInvalidValue && !se2n_diffuse_has(plan->N, P)) return SE2N_EUNSUPPORTED;
    return cuda_status(plan, e);
}

se2n_status fft(se2n_plan *plan, cufftHandle h, float2 *data, int dir) {
    StageTimer timer(plan, SE2N_STAGE_FFT);
    return cufft_status(cufftExecC2C(h, (cufftComplex *)data, (cufftComplex *)data, dir));
}

// The Hermitian-half transforms (in place; the inverse is unnormalised).
se2n_status ensure_half(se2n_plan *plan) {
    if (plan->half_ready) return SE2N_OK;
    int n2[2] = {plan->H, plan->W};
    int real_embed[2] = {plan->H, 2 * plan->Wc};
    int cplx_embed[2] = {plan->H, plan->Wc};
    const int real_dist = plan->H * 2 * plan->Wc, cplx_dist = plan->H * plan->Wc;
    cufftResult r = cufftPlanMany(&plan->fft_r2c, 2, n2, real_embed, 1, real_dist, cplx_embed, 1, cplx_dist, CUFFT_R2C,
                                  plan->N);
    if (r == CUFFT_SUCCESS)
        r = cufftPlanMany(&plan->fft_c2r, 2, n2, cplx_embed, 1, cplx_dist, real_embed, 1, real_dist, CUFFT_C2R,
                          plan->N);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(plan->fft_r2c, plan->stream);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(plan->fft_c2r, plan->stream);
    if (r != CUFFT_SUCCESS) return cufft_status(r);
    plan->half_ready = true;
    return SE2N_OK;
}

se2n_status fft_half(se2n_plan *plan, float2 *data, bool forward) {
    StageTimer timer(plan, SE2N_STAGE_FFT);
    if (forward) return cufft_status(cufftExecR2C(plan->fft_r2c, (cufftReal *)data, (cufftComplex *)data));
    return cufft_status(cufftExecC2R(plan->fft_c2r, (cufftComplex *)data, (cufftReal *)data));
}

se2n_status orient_impl(se2n_plan *plan, const float *f, const uint8_t *mask, double sigma, double flat_tol,
                        uint8_t *bins) {
    if (!(sigma > 0.0) || !(flat_tol >= 0.0) || !isfinite(sigma) || !isfinite(flat_tol)) return SE2N_EINVAL;
    const long long HW = plan->HW;
    float2 *spec = plan->spec;
    StageTimer timer(plan, SE2N_STAGE_ORIENT);
    plan->kernels += 4;
    SE2N_TRY(cuda_status(plan, se2n_launch_orient_prep(f, mask, spec, HW, plan->stream)));
    SE2N_TRY(fft(plan, plan->fft_one, spec, CUFFT_FORWARD));
    SE2N_TRY(cuda_status(plan, se2n_launch_grad_spec(spec, plan->H, plan->W, (float)sigma, plan->stream)));
    SE2N_TRY(fft(plan, plan->fft_two, spec + HW, CUFFT_INVERSE));
    SE2N_TRY(cuda_status(plan, cudaMemsetAsync(plan->gmax, 0, sizeof(unsigned int), plan->stream)));
    SE2N_TRY(cuda_status(plan, se2n_launch_grad_max(spec + HW, spec + 2 * HW, HW, plan->gmax, plan->stream)));
    const float tol2 = (float)(flat_tol * flat_tol);
    return cuda_status(plan, se2n_launch_bins(spec + HW, spec + 2 * HW, HW, plan->gmax, tol2, plan->N,
                                              plan->angle_conv, bins, plan->stream));
}

se2n_status lift_impl(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins, float2 *vol) {
    StageTimer timer(plan, SE2N_STAGE_LIFT);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_lift(f, mask, bins, vol, plan->HW, plan->N, plan->stream));
}

se2n_status mix_impl(se2n_plan *plan, float2 *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                     float scale, float eps, float guard) {
    StageTimer timer(plan, SE2N_STAGE_MIX);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_mix(vol, f, mask, bins, plan->HW, plan->N, scale, eps, guard, plan->stream));
}

se2n_status lift_half_impl(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins, float2 *vol) {
    StageTimer timer(plan, SE2N_STAGE_LIFT);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_lift_r(f, mask, bins, (float *)vol, plan->H, plan->W, plan->N, plan->stream));
}

se2n_status mix_half_impl(se2n_plan *plan, float2 *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                          float scale, float eps, float guard) {
    StageTimer timer(plan, SE2N_STAGE_MIX);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_mix_r((float *)vol, f, mask, bins, plan->H, plan->W, plan->N, scale, eps,
                                               guard, plan->stream));
}

se2n_status project_half_impl(se2n_plan *plan, const float2 *vol, float scale, int proj, const float *f,
                              const uint8_t *mask, float *out) {
    StageTimer timer(plan, SE2N_STAGE_PROJECT);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_project_r((const float *)vol, plan->H, plan->W, plan->N, scale, proj, f, mask,
                                                   out, plan->stream));
}

se2n_status project_impl(se2n_plan *plan, const float2 *vol, float scale, int proj, const float *f,
                         const uint8_t *mask, float *out) {
    StageTimer timer(plan, SE2N_STAGE_PROJECT);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_project(vol, plan->HW, plan->N, scale, proj, f, mask, out, plan->stream));
}

// ---- dynamic restoration (Section 5.3) ----

// One allocation of 12 H W bytes: fref and h (floats), the two good-set
// buffers, bins and the argmax angles (bytes). H W is a multiple of 4, so
// every array is 16-byte aligned.
se2n_status dr_alloc(DrState &d, long long HW) {
    if (d.buf) return SE2N_OK;
    cudaError_t e = cudaMalloc(&d.buf, (size_t)12 * (size_t)HW);
    if (e != cudaSuccess) {
        d.buf = nullptr;
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
    }
    d.fref = (float *)d.buf;
    d.h = (float *)(d.buf + 4 * HW);
    d.mask[0] = d.buf + 8 * HW;
    d.mask[1] = d.buf + 9 * HW;
    d.bins = d.buf + 10 * HW;
    d.amax = d.buf + 11 * HW;
    d.cur = 0;
    return SE2N_OK;
}

void dr_free(DrState &d) {
    cudaFree(d.buf);
    d = DrState();
}

// Start of an inpaint: the good set is the known pixels, each referenced to
// its value in f at its orientation bin.
se2n_status dr_begin(se2n_plan *plan, DrState &d, const float *f, const uint8_t *mask, const uint8_t *bins) {
    const size_t HW = (size_t)plan->HW;
    cudaError_t e = cudaMemcpyAsync(d.fref, f, 4 * HW, cudaMemcpyDeviceToDevice, plan->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.mask[0], mask, HW, cudaMemcpyDeviceToDevice, plan->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.bins, bins, HW, cudaMemcpyDeviceToDevice, plan->stream);
    d.cur = 0;
    return cuda_status(plan, e);
}

// One growth step from the (unnormalised, times scale) volume.
se2n_status dr_step(se2n_plan *plan, DrState &d, const float2 *vol, float scale, bool half) {
    StageTimer timer(plan, SE2N_STAGE_DR);
    plan->kernels += 2;
    cudaError_t e = half ? se2n_launch_dr_max_r((const float *)vol, plan->H, plan->W, plan->N, scale, d.h, d.amax,
                                                plan->stream)
                         : se2n_launch_dr_max(vol, plan->HW, plan->N, scale, d.h, d.amax, plan->stream);
    if (e == cudaSuccess)
        e = se2n_launch_dr_grow(d.h, d.amax, d.mask[d.cur], d.mask[d.cur ^ 1], d.fref, d.bins, plan->H, plan->W,
                                plan->stream);
    d.cur ^= 1;
    return cuda_status(plan, e);
}

// The growth step itself, from h and amax already in d (the row pass with
// SE2N_ROW_OUT_H computes them).
se2n_status dr_grow_only(se2n_plan *plan, DrState &d) {
    StageTimer timer(plan, SE2N_STAGE_DR);
    plan->kernels += 1;
    const cudaError_t e = se2n_launch_dr_grow(d.h, d.amax, d.mask[d.cur], d.mask[d.cur ^ 1], d.fref, d.bins, plan->H,
                                              plan->W, plan->stream);
    d.cur ^= 1;
    return cuda_status(plan, e);
}

// The restoration at the end of an interval: static on (f, mask, bins), or,
// with dr, one growth step of the good set and then the static restoration
// towards the references of the grown set.
se2n_status restore_impl(se2n_plan *plan, DrState *dr, float2 *vol, const float *f, const uint8_t *mask,
                         const uint8_t *bins, float scale, float eps, float guard, bool half) {
    if (dr) {
        SE2N_TRY(dr_step(plan, *dr, vol, scale, half));
        f = dr->fref;
        mask = dr->mask[dr->cur];
        bins = dr->bins;
    }
    return half ? mix_half_impl(plan, vol, f, mask, bins, scale, eps, guard)
                : mix_impl(plan, vol, f, mask, bins, scale, eps, guard);
}

se2n_status check_params(const se2n_plan *plan, const se2n_params *p) {
    if (!p) return SE2N_EINVAL;
    if (p->N != plan->N || !(p->beta > 0.0) || !(p->T >= 0.0) || p->steps < 1 || p->rounds < 1) return SE2N_EINVAL;
    if (!(p->eps >= 0.0 && p->eps <= 1.0) || !(p->sigma_smooth > 0.0) || !(p->flat_tol >= 0.0)) return SE2N_EINVAL;
    if ((p->proj != SE2N_PROJ_MAX && p->proj != SE2N_PROJ_MEAN) || (p->final_mix != 0 && p->final_mix != 1) ||
        (p->reinject != 0 && p->reinject != 1) || (p->full_spectrum != 0 && p->full_spectrum != 1) ||
        (p->dynamic != 0 && p->dynamic != 1))
        return SE2N_EINVAL;
    if (!(p->guard >= 0.0) || (p->diffuse_flags & ~(SE2N_DIFFUSE_SM_FP64 | SE2N_DIFFUSE_SPLIT_DIAG |
                                                    SE2N_DIFFUSE_FULL_CORRECTION | SE2N_DIFFUSE_PROPAGATOR)))
        return SE2N_EINVAL;
    if (!isfinite(p->beta) || !isfinite(p->T) || !isfinite(p->sigma_smooth) || !isfinite(p->guard))
        return SE2N_EINVAL;
    if (p->T > 0.0) {
        const double bdt = p->beta * (p->T / p->rounds) / p->steps;
        if (!(bdt >= 1e-30 && bdt <= 1e3)) return SE2N_ENUMERIC;
    }
    return SE2N_OK;
}

// allow_col = false keeps the separate transforms and propagator apply (the
// path the batch graph takes, so that its per-image replay gives its bits).
se2n_status inpaint_impl(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins_in,
                         const se2n_params *p, float2 *vol, float *out, bool allow_col = true) {
    const long long HW = plan->HW;
    const int N = plan->N;
    const uint8_t *bins = bins_in;
    const bool col = allow_col && col_path(plan, p);
    if (col) SE2N_TRY(col_start(plan, p));
    if (!bins) {
        SE2N_TRY(orient_impl(plan, f, mask, p->sigma_smooth, p->flat_tol, plan->bins));
        bins = plan->bins;
    }
    const double Tr = p->T / p->rounds;
    const float inv_hw = (float)(1.0 / (double)HW);
    const float eps = (float)p->eps, guard = (float)p->guard;
    DrState *dr = nullptr;
    if (p->dynamic) {
        SE2N_TRY(dr_alloc(plan->dr, HW));
        dr = &plan->dr;
        SE2N_TRY(dr_begin(plan, *dr, f, mask, bins));
    }
    if (!p->full_spectrum) {
        // The lifted volume is real, so its spectrum is Hermitian and the
        // system of frequency (-k, -l) is that of (k, l) conjugated (a_r^2 is
        // even in the frequency): integrate the half l = 0 .. W/2 only, with
        // real-to-complex transforms, and let the inverse transform rebuild
        // the rest.
        if (col) {
            // With propagators on a supported shape the volume stays
            // row-transformed between intervals: a row pass (lift, or
            // inverse DFT along x, restoration and forward DFT along x) and
            // a column pass (DFT along y, propagators, inverse DFT along y)
            // an interval, the projection fused into the last row pass.
            // Dynamic restoration adds a row pass that gives the image
            // value and its argmax angle before each growth step.
            RowArgs r = row_args(plan, f, mask, bins, inv_hw, eps, guard);
            r.in_mode = SE2N_ROW_IN_LIFT;
            SE2N_TRY(row_pass(plan, r));
            SE2N_TRY(col_diffuse(plan, p->beta, Tr, p->steps));
            for (int i = 1; i <= p->rounds; ++i) {
                const bool last = i == p->rounds;
                const float *rf = f;
                const uint8_t *rmask = mask, *rbins = bins;
                if (dr && (!last || p->final_mix)) {
                    // a growth step: the image value h and its argmax angle
                    // from one row pass, then the set grows; the restoration
                    // below pulls the grown set to its references
                    r = row_args(plan, f, mask, bins, inv_hw, eps, guard);
                    r.out_mode = SE2N_ROW_OUT_H;
                    r.h_out = dr->h;
                    r.amax_out = dr->amax;
                    SE2N_TRY(row_pass(plan, r));
                    SE2N_TRY(dr_grow_only(plan, *dr));
                    rf = dr->fref;
                    rmask = dr->mask[dr->cur];
                    rbins = dr->bins;
                }
                r = row_args(plan, rf, rmask, rbins, inv_hw, eps, guard);
                r.rf = f;     // reinjection keeps the given known pixels
                r.rmask = mask;
                if (last) {
                    r.mix = p->final_mix;
                    r.out_mode = SE2N_ROW_OUT_PROJ;
                    r.proj_out = out;
                    r.proj = p->proj;
                    r.reinject = p->reinject;
                    r.scale_proj = p->final_mix ? 1.0f : inv_hw;
                    return row_pass(plan, r);
                }
                r.mix = 1;
                SE2N_TRY(row_pass(plan, r));
                SE2N_TRY(col_diffuse(plan, p->beta, Tr, p->steps));
            }
        } else {
            SE2N_TRY(ensure_half(plan));
            SE2N_TRY(lift_half_impl(plan, f, mask, bins, vol));
            SE2N_TRY(fft_half(plan, vol, true));
            SE2N_TRY(diffuse_impl(plan, vol, p->beta, Tr, p->steps, p->diffuse_flags, true));
            for (int i = 1; i < p->rounds; ++i) {
                SE2N_TRY(fft_half(plan, vol, false));
                SE2N_TRY(restore_impl(plan, dr, vol, f, mask, bins, inv_hw, eps, guard, true));
                SE2N_TRY(fft_half(plan, vol, true));
                SE2N_TRY(diffuse_impl(plan, vol, p->beta, Tr, p->steps, p->diffuse_flags, true));
            }
            SE2N_TRY(fft_half(plan, vol, false));
        }
        float scale = inv_hw;
        if (p->final_mix) {
            SE2N_TRY(restore_impl(plan, dr, vol, f, mask, bins, inv_hw, eps, guard, true));
            scale = 1.0f;
        }
        return project_half_impl(plan, vol, scale, p->proj, p->reinject ? f : nullptr, p->reinject ? mask : nullptr,
                                 out);
    }
    SE2N_TRY(lift_impl(plan, f, mask, bins, vol));
    SE2N_TRY(fft(plan, plan->fft_vol, vol, CUFFT_FORWARD));
    SE2N_TRY(diffuse_impl(plan, vol, p->beta, Tr, p->steps, p->diffuse_flags));
    for (int i = 1; i < p->rounds; ++i) {
        // inverse DFT; its 1/(H W) is folded into the restoration kernel
        SE2N_TRY(fft(plan, plan->fft_vol, vol, CUFFT_INVERSE));
        SE2N_TRY(restore_impl(plan, dr, vol, f, mask, bins, inv_hw, eps, guard, false));
        SE2N_TRY(fft(plan, plan->fft_vol, vol, CUFFT_FORWARD));
        SE2N_TRY(diffuse_impl(plan, vol, p->beta, Tr, p->steps, p->diffuse_flags));
    }
    SE2N_TRY(fft(plan, plan->fft_vol, vol, CUFFT_INVERSE));
    float scale = inv_hw;
    if (p->final_mix) {
        SE2N_TRY(restore_impl(plan, dr, vol, f, mask, bins, inv_hw, eps, guard, false));
        scale = 1.0f;
    }
    return project_impl(plan, vol, scale, p->proj, p->reinject ? f : nullptr, p->reinject ? mask : nullptr, out);
}

void free_plan(se2n_plan *plan) {
    if (plan->fft_vol) cufftDestroy(plan->fft_vol);
    if (plan->fft_one) cufftDestroy(plan->fft_one);
    if (plan->fft_two) cufftDestroy(plan->fft_two);
    if (plan->fft_r2c) cufftDestroy(plan->fft_r2c);
    if (plan->fft_c2r) cufftDestroy(plan->fft_c2r);
    if (plan->side) {
        cudaStreamSynchronize(plan->side);
        cudaStreamDestroy(plan->side);
        cudaEventDestroy(plan->ev_fork);
        cudaEventDestroy(plan->ev_join);
    }
    cudaFree(plan->colbuf);
    cudaFree(plan->col_tw);
    cudaFree(plan->row_tw);
    cudaFree(plan->spec);
    cudaFree(plan->gmax);
    cudaFree(plan->bins);
    cudaFree(plan->h_f);
    cudaFree(plan->h_out);
    cudaFree(plan->h_mask);
    cudaFree(plan->h_vol);
    dr_free(plan->dr);
    cudaFree(plan->prop_D);
    for (int st = 0; st < SE2N_NUM_STAGES; ++st)
        for (cudaEvent_t e : plan->stage_ev[st]) cudaEventDestroy(e);
    delete plan;
}

}  // namespace

extern "C" {

const char *se2n_status_string(se2n_status s) {
    switch (s) {
        case SE2N_OK: return "SE2N_OK";
        case SE2N_EINVAL: return "SE2N_EINVAL: invalid argument";
        case SE2N_ENOMEM: return "SE2N_ENOMEM: allocation failed";
        case SE2N_ECUDA: return "SE2N_ECUDA: CUDA error";
        case SE2N_ECUFFT: return "SE2N_ECUFFT: cuFFT error";
        case SE2N_EUNSUPPORTED: return "SE2N_EUNSUPPORTED: no kernel for this configuration";
        case SE2N_ENUMERIC: return "SE2N_ENUMERIC: beta*dt outside the range the FP32 scheme resolves";
    }
    return "SE2N: unknown status";
}

se2n_status se2n_params_default(se2n_params *p) {
    if (!p) return SE2N_EINVAL;
    p->N = 32;
    p->beta = 0.25;
    p->T = 2.0;
    p->steps = 100;
    p->rounds = 1;
    p->eps = 0.5;
    p->sigma_smooth = 1.0;
    p->flat_tol = 1e-4;
    p->proj = SE2N_PROJ_MAX;
    p->final_mix = 0;
    p->guard = 0.1;
    p->diffuse_flags = 0;
    p->reinject = 0;
    p->full_spectrum = 0;
    p->dynamic = 0;
    return SE2N_OK;
}

se2n_status se2n_params_from_paper(double alpha, double T_paper, int M, int N, double *beta_out,
                                   double *T_out) {
    if (!beta_out || !T_out || M < 2 || N < 3 || !(alpha >= 0.0) || !(T_paper >= 0.0)) return SE2N_EINVAL;
    const double beta_N = alpha * (N / (2.0 * kPi)) * (N / (2.0 * kPi));
    *beta_out = beta_N / M;
    *T_out = 0.5 * M * T_paper;
    return SE2N_OK;
}

se2n_status se2n_plan_create(se2n_plan **out, int H, int W, int N, int angle_conv, void *stream) {
    if (!out || H < 2 || W < 2 || (H % 2) || (W % 2)) return SE2N_EINVAL;
    if ((long long)H * W > (1LL << 28)) return SE2N_EINVAL;
    if (N < 3 || N > SE2N_MAX_N || (angle_conv != 0 && angle_conv != 1)) return SE2N_EINVAL;
    if (!se2n_diffuse_has(N, se2n_diffuse_default_P(N))) return SE2N_EUNSUPPORTED;
    se2n_plan *plan = new (std::nothrow) se2n_plan();
    if (!plan) return SE2N_ENOMEM;
    plan->H = H;
    plan->W = W;
    plan->N = N;
    plan->angle_conv = angle_conv;
    plan->HW = (long long)H * W;
    plan->Wc = W / 2 + 1;
    plan->fft_r2c = 0;
    plan->fft_c2r = 0;
    plan->half_ready = false;
    plan->stream = (cudaStream_t)stream;
    plan->diffuse_P = se2n_diffuse_default_P(N);
    plan->diffuse_block = 0;
    plan->diffuse_blocks = 0;
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&plan->num_sms, cudaDevAttrMultiProcessorCount, plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return SE2N_ECUDA;
    }
    int n2[2] = {H, W};
    cufftResult r = cufftPlanMany(&plan->fft_vol, 2, n2, nullptr, 1, (int)plan->HW, nullptr, 1, (int)plan->HW,
                                  CUFFT_C2C, N);
    if (r == CUFFT_SUCCESS) r = cufftPlan2d(&plan->fft_one, H, W, CUFFT_C2C);
    if (r == CUFFT_SUCCESS)
        r = cufftPlanMany(&plan->fft_two, 2, n2, nullptr, 1, (int)plan->HW, nullptr, 1, (int)plan->HW, CUFFT_C2C, 2);
    if (r != CUFFT_SUCCESS) {
        free_plan(plan);
        return cufft_status(r);
    }
    e = cudaMalloc(&plan->spec, sizeof(float2) * 3 * plan->HW);
    if (e == cudaSuccess) e = cudaMalloc(&plan->gmax, 256);
    if (e == cudaSuccess) e = cudaMalloc(&plan->bins, plan->HW);
    if (e != cudaSuccess) {
        free_plan(plan);
        return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
    }
    if (cufftSetStream(plan->fft_vol, plan->stream) != CUFFT_SUCCESS ||
        cufftSetStream(plan->fft_one, plan->stream) != CUFFT_SUCCESS ||
        cufftSetStream(plan->fft_two, plan->stream) != CUFFT_SUCCESS) {
        free_plan(plan);
        return SE2N_ECUFFT;
    }
    *out = plan;
    return SE2N_OK;
}

se2n_status se2n_plan_destroy(se2n_plan *plan) {
    if (!plan) return SE2N_OK;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    return SE2N_OK;
}

se2n_status se2n_plan_set_stream(se2n_plan *plan, void *stream) {
    SE2N_TRY(check_plan(plan));
    cudaStream_t s = (cudaStream_t)stream;
    if (cufftSetStream(plan->fft_vol, s) != CUFFT_SUCCESS || cufftSetStream(plan->fft_one, s) != CUFFT_SUCCESS ||
        cufftSetStream(plan->fft_two, s) != CUFFT_SUCCESS)
        return SE2N_ECUFFT;
    if (plan->half_ready &&
        (cufftSetStream(plan->fft_r2c, s) != CUFFT_SUCCESS || cufftSetStream(plan->fft_c2r, s) != CUFFT_SUCCESS))
        return SE2N_ECUFFT;
    plan->stream = s;
    return SE2N_OK;
}

int se2n_plan_last_cuda_error(const se2n_plan *plan) { return plan ? plan->last_cuda_error : 0; }

se2n_status se2n_orient(se2n_plan *plan, const float *f, const uint8_t *mask, double sigma, double flat_tol,
                        uint8_t *bins) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(f, 8) || !device_ptr(mask, 2) || !device_ptr(bins, 2)) return SE2N_EINVAL;
    return orient_impl(plan, f, mask, sigma, flat_tol, bins);
}

se2n_status se2n_lift(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins, void *vol) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(f, 8) || !device_ptr(mask, 2) || !device_ptr(bins, 2) || !device_ptr(vol, 16))
        return SE2N_EINVAL;
    return lift_impl(plan, f, mask, bins, (float2 *)vol);
}

se2n_status se2n_forward(se2n_plan *plan, void *vol) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol, 16)) return SE2N_EINVAL;
    return fft(plan, plan->fft_vol, (float2 *)vol, CUFFT_FORWARD);
}

se2n_status se2n_inverse(se2n_plan *plan, void *vol) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol, 16)) return SE2N_EINVAL;
    SE2N_TRY(fft(plan, plan->fft_vol, (float2 *)vol, CUFFT_INVERSE));
    StageTimer timer(plan, SE2N_STAGE_FFT);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_scale((float2 *)vol, plan->HW * plan->N, (float)(1.0 / (double)plan->HW),
                                               plan->stream));
}

se2n_status se2n_diffuse(se2n_plan *plan, void *vol_hat, double beta, double T, int steps, int flags) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol_hat, 16)) return SE2N_EINVAL;
    return diffuse_impl(plan, (float2 *)vol_hat, beta, T, steps, flags);
}

se2n_status se2n_diffuse_rows(se2n_plan *plan, void *vol_rows, int k0, int rows, double beta, double T, int steps,
                              int flags) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol_rows, 16) || k0 < 0 || rows < 1 || k0 + rows > plan->H) return SE2N_EINVAL;
    return diffuse_impl(plan, (float2 *)vol_rows, beta, T, steps, flags, false, k0, rows);
}

se2n_status se2n_dr_grow(se2n_plan *plan, const void *vol, const uint8_t *mask_in, uint8_t *mask_out, float *fref,
                         uint8_t *bins) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol, 16) || !device_ptr(mask_in, 1) || !device_ptr(mask_out, 1) || !device_ptr(fref, 4) ||
        !device_ptr(bins, 1))
        return SE2N_EINVAL;
    const uintptr_t a = (uintptr_t)mask_in, o = (uintptr_t)mask_out, HW = (uintptr_t)plan->HW;
    if (a < o + HW && o < a + HW) return SE2N_EINVAL;  // the step reads the old set while writing the new one
    SE2N_TRY(dr_alloc(plan->dr, plan->HW));  // h and the argmax angles
    DrState &d = plan->dr;
    StageTimer timer(plan, SE2N_STAGE_DR);
    plan->kernels += 2;
    cudaError_t e = se2n_launch_dr_max((const float2 *)vol, plan->HW, plan->N, 1.0f, d.h, d.amax, plan->stream);
    if (e == cudaSuccess)
        e = se2n_launch_dr_grow(d.h, d.amax, mask_in, mask_out, fref, bins, plan->H, plan->W, plan->stream);
    return cuda_status(plan, e);
}

se2n_status se2n_mix(se2n_plan *plan, void *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                     double eps, double guard) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol, 16) || !device_ptr(f, 8) || !device_ptr(mask, 2) || !device_ptr(bins, 2))
        return SE2N_EINVAL;
    if (!(eps >= 0.0 && eps <= 1.0) || !(guard >= 0.0) || !isfinite(guard)) return SE2N_EINVAL;
    return mix_impl(plan, (float2 *)vol, f, mask, bins, 1.0f, (float)eps, (float)guard);
}

se2n_status se2n_mix_given(se2n_plan *plan, void *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                           const float *h_t, double eps, double guard) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol, 16) || !device_ptr(f, 8) || !device_ptr(mask, 2) || !device_ptr(bins, 2) ||
        !device_ptr(h_t, 8))
        return SE2N_EINVAL;
    if (!(eps >= 0.0 && eps <= 1.0) || !(guard >= 0.0) || !isfinite(guard)) return SE2N_EINVAL;
    StageTimer timer(plan, SE2N_STAGE_MIX);
    plan->kernels += 1;
    return cuda_status(plan, se2n_launch_mix_given((float2 *)vol, f, mask, bins, h_t, plan->HW, plan->N,
                                                   (float)eps, (float)guard, plan->stream));
}

se2n_status se2n_project(se2n_plan *plan, const void *vol, int proj, float *out) {
    SE2N_TRY(check_plan(plan));
    if (!device_ptr(vol, 16) || !device_ptr(out, 8)) return SE2N_EINVAL;
    if (proj != SE2N_PROJ_MAX && proj != SE2N_PROJ_MEAN) return SE2N_EINVAL;
    return project_impl(plan, (const float2 *)vol, 1.0f, proj, nullptr, nullptr, out);
}

se2n_status se2n_inpaint(se2n_plan *plan, const float *f, const uint8_t *mask, const uint8_t *bins_in,
                         const se2n_params *p, void *vol, float *out) {
    SE2N_TRY(check_plan(plan));
    SE2N_TRY(check_params(plan, p));
    if (!device_ptr(f, 8) || !device_ptr(mask, 2) || !device_ptr(vol, 16) || !device_ptr(out, 8)) return SE2N_EINVAL;
    if (bins_in && !device_ptr(bins_in, 2)) return SE2N_EINVAL;
    return inpaint_impl(plan, f, mask, bins_in, p, (float2 *)vol, out);
}

se2n_status se2n_inpaint_host(se2n_plan *plan, const float *f_host, const uint8_t *mask_host,
                              const se2n_params *p, float *out_host) {
    SE2N_TRY(check_plan(plan));
    SE2N_TRY(check_params(plan, p));
    if (!f_host || !mask_host || !out_host) return SE2N_EINVAL;
    const long long HW = plan->HW;
    if (!plan->h_vol) {
        cudaError_t e = cudaMalloc(&plan->h_vol, sizeof(float2) * HW * plan->N);
        if (e == cudaSuccess) e = cudaMalloc(&plan->h_f, sizeof(float) * HW);
        if (e == cudaSuccess) e = cudaMalloc(&plan->h_out, sizeof(float) * HW);
        if (e == cudaSuccess) e = cudaMalloc(&plan->h_mask, HW);
        if (e != cudaSuccess) {
            cudaFree(plan->h_vol);
            cudaFree(plan->h_f);
            cudaFree(plan->h_out);
            cudaFree(plan->h_mask);
            plan->h_vol = nullptr;
            plan->h_f = plan->h_out = nullptr;
            plan->h_mask = nullptr;
            return cuda_status(plan, e);
        }
    }
    if (col_path(plan, p)) SE2N_TRY(col_start(plan, p));  // the build overlaps the copies too
    SE2N_TRY(cuda_status(plan, cudaMemcpyAsync(plan->h_f, f_host, sizeof(float) * HW, cudaMemcpyHostToDevice,
                                               plan->stream)));
    SE2N_TRY(cuda_status(plan, cudaMemcpyAsync(plan->h_mask, mask_host, HW, cudaMemcpyHostToDevice, plan->stream)));
    SE2N_TRY(inpaint_impl(plan, plan->h_f, plan->h_mask, nullptr, p, plan->h_vol, plan->h_out));
    SE2N_TRY(cuda_status(plan, cudaMemcpyAsync(out_host, plan->h_out, sizeof(float) * HW, cudaMemcpyDeviceToHost,
                                               plan->stream)));
    return cuda_status(plan, cudaStreamSynchronize(plan->stream));
}

se2n_status se2n_plan_drop_propagators(se2n_plan *plan, int free_memory) {
    SE2N_TRY(check_plan(plan));
    plan->prop_valid = false;
    if (free_memory && plan->prop_D) {
        prop_join(plan);  // a build still running on the side stream
        SE2N_TRY(cuda_status(plan, cudaStreamSynchronize(plan->stream)));
        cudaFree(plan->prop_D);
        plan->prop_D = nullptr;
        plan->prop_bytes = 0;
    }
    return SE2N_OK;
}

se2n_status se2n_plan_tune_diffuse(se2n_plan *plan, int threads_per_freq, int block_threads, int blocks) {
    SE2N_TRY(check_plan(plan));
    const int P = threads_per_freq ? threads_per_freq : se2n_diffuse_default_P(plan->N);
    const int block = block_threads;
    if (P != 1 && P != 2 && P != 4) return SE2N_EINVAL;
    if (block < 0 || block > 384 || (block % 32) || blocks < 0) return SE2N_EINVAL;
    if (!se2n_diffuse_has(plan->N, P)) return SE2N_EUNSUPPORTED;
    plan->diffuse_P = P;
    plan->diffuse_block = block;
    plan->diffuse_blocks = blocks;
    return SE2N_OK;
}

se2n_status se2n_plan_diffuse_info(se2n_plan *plan, int *regs_per_thread, int *blocks_per_sm,
                                   int *threads_per_freq) {
    SE2N_TRY(check_plan(plan));
    int regs = 0, per_sm = 0, block = 0, blocks = 0;
    cudaError_t e = se2n_diffuse_shape(plan->N, plan->diffuse_P, false, false, true, plan->diffuse_block,
                                       plan->diffuse_blocks, plan->num_sms, plan->HW, &block, &blocks);
    if (e == cudaSuccess)
        e = se2n_diffuse_occupancy(plan->N, plan->diffuse_P, false, false, true, block, &per_sm, &regs);
    if (e != cudaSuccess) return cuda_status(plan, e);
    if (regs_per_thread) *regs_per_thread = regs;
    if (blocks_per_sm) *blocks_per_sm = per_sm;
    if (threads_per_freq) *threads_per_freq = plan->diffuse_P;
    return SE2N_OK;
}

se2n_status se2n_plan_profile(se2n_plan *plan, int enable) {
    SE2N_TRY(check_plan(plan));
    SE2N_TRY(cuda_status(plan, cudaStreamSynchronize(plan->stream)));
    plan->profiling = enable != 0;
    for (int st = 0; st < SE2N_NUM_STAGES; ++st) {
        plan->stage_used[st] = 0;
        plan->prof_ms[st] = 0.0;
        plan->prof_calls[st] = 0;
    }
    plan->kernels = 0;
    return SE2N_OK;
}

se2n_status se2n_plan_profile_read(se2n_plan *plan, se2n_profile *out, int reset) {
    SE2N_TRY(check_plan(plan));
    if (!out) return SE2N_EINVAL;
    SE2N_TRY(cuda_status(plan, cudaStreamSynchronize(plan->stream)));
    for (int st = 0; st < SE2N_NUM_STAGES; ++st) {
        for (int i = 0; i < plan->stage_used[st]; ++i) {
            float ms = 0.0f;
            cudaError_t e = cudaEventElapsedTime(&ms, plan->stage_ev[st][2 * i], plan->stage_ev[st][2 * i + 1]);
            if (e != cudaSuccess) return cuda_status(plan, e);
            plan->prof_ms[st] += ms;
        }
        plan->prof_calls[st] += plan->stage_used[st];
        plan->stage_used[st] = 0;
        out->ms[st] = plan->prof_ms[st];
        out->calls[st] = plan->prof_calls[st];
    }
    out->kernels = plan->kernels;
    if (reset) {
        for (int st = 0; st < SE2N_NUM_STAGES; ++st) {
            plan->prof_ms[st] = 0.0;
            plan->prof_calls[st] = 0;
        }
        plan->kernels = 0;
    }
    return SE2N_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------

struct se2n_batch {
    int count = 0, angle_conv = 0, device = 0;
    cudaStream_t stream = nullptr;
    se2n_params p{};
    std::vector<se2n_image_desc> imgs;
    std::vector<se2n_plan *> plans;    // owned, one per distinct (H, W, N)
    std::vector<se2n_plan *> plan_of;  // per image
    char *arena = nullptr;
    size_t vol_bytes = 0;
    std::vector<float2 *> vols;
    std::vector<uint8_t *> bins;
    std::vector<DrState> dr;  // per image, with dynamic restoration
    std::vector<char> img_prop;   // per image: integrated by its shape's propagators
    std::vector<char> img_fused;  // per image: the whole inpaint on the row and column passes
    int prop_images = 0, fused_images = 0;
    std::vector<BatchImage> h_imgs;
    float *d_tables = nullptr;
    BatchImage *d_imgs = nullptr;
    BatchItem *d_items = nullptr;
    size_t items_cap = 0;
    unsigned int *d_counter = nullptr;
    int n_items = 0, config = 0, passes = 8, block = 256, blocks = 0;
    bool fast = false, split = false;
    int candidates = 0;
    double best_ms = 0.0, worst_ms = 0.0, updates = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int num_sms = 0;
    bool flags_autotune = false;
    bool own_stream = false;  // created because the caller passed the legacy stream
};

namespace {

std::vector<BatchItem> build_items(const se2n_batch *b, int config, int passes) {
    std::vector<int> order(b->count);
    for (int i = 0; i < b->count; ++i) order[i] = i;
    // costliest first: larger N, then larger images
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const se2n_image_desc &a = b->imgs[x], &c = b->imgs[y];
        if (a.N != c.N) return a.N > c.N;
        return (long long)a.H * a.W > (long long)c.H * c.W;
    });
    std::vector<BatchItem> items;
    for (int i : order) {
        if (!b->img_prop.empty() && b->img_prop[i]) continue;  // integrated by propagators
        const se2n_image_desc &d = b->imgs[i];
        const long long HW = b->h_imgs[i].HW;  // frequencies integrated (the Hermitian half by default)
        const int per = 32 / se2n_batch_config_P(config, d.N);
        const long long tile = (long long)per * passes;
        for (long long f0 = 0; f0 < HW; f0 += tile) {
            BatchItem it;
            it.image = i;
            it.first = f0;
            it.count = (int)std::min(tile, HW - f0);
            items.push_back(it);
        }
    }
    return items;
}

se2n_status upload_items(se2n_batch *b, const std::vector<BatchItem> &items) {
    if (items.size() > b->items_cap) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        cudaError_t e = cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size());
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
        b->items_cap = items.size();
    }
    cudaError_t e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->n_items = (int)items.size();
    return e == cudaSuccess ? SE2N_OK : SE2N_ECUDA;
}

se2n_status batch_diffuse(se2n_batch *b, int steps, double T) {
    const double dt = T / steps;
    const StepParams sp = step_params(b->p.beta, b->p.beta * dt, steps);
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess)
        e = se2n_launch_diffuse_batch(b->config, b->fast, b->split, sp, b->d_tables, b->d_imgs, b->d_items,
                                      b->n_items, b->d_counter, b->block, b->blocks, b->stream);
    return e == cudaSuccess ? SE2N_OK : SE2N_ECUDA;
}

// One interval of every image: the persistent step-by-step launch over the
// whole batch, or, with SE2N_DIFFUSE_PROPAGATOR, each image's propagators
// (built once per distinct plan shape, which the images of that shape share).
se2n_status batch_interval(se2n_batch *b, double Tr, bool half) {
    const se2n_params &p = b->p;
    if (b->prop_images < b->count) SE2N_TRY(batch_diffuse(b, p.steps, Tr));
    if (b->prop_images > 0)
        for (int i = 0; i < b->count; ++i)
            if (b->img_prop[i] && !b->img_fused[i])
                SE2N_TRY(diffuse_impl(b->plan_of[i], b->vols[i], p.beta, Tr, p.steps, p.diffuse_flags, half));
    return SE2N_OK;
}

// With SE2N_DIFFUSE_PROPAGATOR, the images of one shape are integrated by
// that shape's propagators when building them once and applying them to every
// image and interval is estimated to cost less than the step-by-step kernel on
// those images. The estimate uses this library's measured rates on a GB300:
// the step kernel about 54 TFLOP/s at 22 flops an update; the build about
// 22 TFLOP/s (N = 16, 32) and 28 TFLOP/s (N = 64) of the flops it executes
// (the powering program's products, 2 N^3 flops each, on the 3 of 4, 10 of
// 16 or 36 of 64 upper-triangle tiles, for the classes it builds: half of
// them on square planes of the Hermitian half, whose transposed classes
// share a build); the apply about 2 TB/s.
void choose_propagators(se2n_batch *b) {
    const se2n_params &p = b->p;
    b->img_prop.assign(b->count, 0);
    b->img_fused.assign(b->count, 0);
    b->prop_images = 0;
    b->fused_images = 0;
    if (!(p.diffuse_flags & SE2N_DIFFUSE_PROPAGATOR)) return;
    if (!prop_admissible(p.beta, p.T / p.rounds / p.steps)) return;
    const bool half = !p.full_spectrum;
    const int S = p.steps;
    unsigned char ops[SE2N_PROP_CHAIN_MAX];
    int len = 0, in_r = 0, products = 0;
    if (se2n_prop_chain(S, ops, SE2N_PROP_CHAIN_MAX, &len, &in_r) != SE2N_OK) return;
    for (int o = 0; o < len; ++o) products += ops[o] != PROP_COPY;
    for (se2n_plan *pl : b->plans) {
        int n_img = 0;
        for (int i = 0; i < b->count; ++i) n_img += b->plan_of[i] == pl;
        const double freqs = (double)pl->H * (half ? pl->W / 2 + 1 : pl->W);
        const double N = se2n_prop_dim(pl->N);
        const double steps_s = n_img * (double)p.rounds * freqs * pl->N * S * 22.0 / 54e12;
        const double classes = (double)se2n_prop_classes(pl->H, pl->W, half);
        const bool share_t = half && pl->H == pl->W && (pl->angle_conv == 0 || pl->N % 4 == 0);
        const double built = share_t ? classes * 0.5 : classes;
        const double tiles = N == 16 ? 3.0 / 4.0 : (N == 32 ? 10.0 / 16.0 : 36.0 / 64.0);
        const double build_s = built * products * 2.0 * N * N * N * tiles / (N == 64 ? 28e12 : 22e12);
        // the apply: by diagonals (about 2 TB/s), or tile by tile from the
        // built classes' rows (N = 64 on the half: 3.05 TB/s measured at 1024 x 1024)
        const double apply_s =
            se2n_prop_apply_fmt(pl->N, half) == PROP_ROWS
                ? n_img * (double)p.rounds * (built * 4.0 * N * N + 16.0 * freqs * N) / 3e12
                : n_img * (double)p.rounds * (classes * 4.0 * N * (N / 2 + 1) + 16.0 * freqs * N) / 2e12;
        if (build_s + apply_s < steps_s) {
            // shapes the row and column passes cover take them (whole inpaints)
            const bool fused = col_path(pl, &p);
            for (int i = 0; i < b->count; ++i)
                if (b->plan_of[i] == pl) {
                    b->img_prop[i] = 1;
                    b->prop_images += 1;
                    b->img_fused[i] = fused;
                    b->fused_images += fused;
                }
        }
    }
}

se2n_status set_shape(se2n_batch *b, int config, int passes, int block) {
    int per_sm = 0;
    if (se2n_batch_occupancy(config, b->fast, b->split, block, &per_sm) != cudaSuccess) return SE2N_ECUDA;
    b->config = config;
    b->passes = passes;
    b->block = block;
    b->blocks = b->num_sms * std::max(per_sm, 1);
    return upload_items(b, build_items(b, config, passes));
}

// Time every candidate launch shape on this batch (diffusion only, a few
// steps, on zeroed volumes that the graph's lift overwrites later) and keep
// the fastest.
se2n_status autotune(se2n_batch *b) {
    const int steps = std::min(b->p.steps, 16);
    const double T = b->p.T / b->p.rounds * steps / b->p.steps;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SE2N_ECUDA;
    double best = 1e30, worst = 0.0;
    int bc = 0, bp = 8, bb = 256;
    const int passes_c[] = {2, 8, 32};
    const int block_c[] = {128, 256};
    se2n_status st = SE2N_OK;
    for (int c = 0; c < se2n_batch_configs() && st == SE2N_OK; ++c)
        for (int pc : passes_c)
            for (int bl : block_c) {
                st = set_shape(b, c, pc, bl);
                if (st != SE2N_OK) break;
                st = batch_diffuse(b, steps, T);  // warm
                cudaEventRecord(e0, b->stream);
                if (st == SE2N_OK) st = batch_diffuse(b, steps, T);
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = SE2N_ECUDA;
                if (st != SE2N_OK) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                b->candidates += 1;
                worst = std::max(worst, (double)ms);
                if (ms < best) {
                    best = ms;
                    bc = c;
                    bp = pc;
                    bb = bl;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SE2N_OK) return st;
    b->best_ms = best;
    b->worst_ms = worst;
    return set_shape(b, bc, bp, bb);
}

se2n_status enqueue_batch_half(se2n_batch *b) {
    const se2n_params &p = b->p;
    const double Tr = p.T / p.rounds;
    for (int i = 0; i < b->count; ++i) {
        se2n_plan *pl = b->plan_of[i];
        const se2n_image_desc &d = b->imgs[i];
        if (d.bins) {
            if (cudaMemcpyAsync(b->bins[i], d.bins, (size_t)pl->HW, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
                return SE2N_ECUDA;
        } else {
            SE2N_TRY(orient_impl(pl, d.f, d.mask, p.sigma_smooth, p.flat_tol, b->bins[i]));
        }
        if (b->img_fused[i]) continue;
        SE2N_TRY(lift_half_impl(pl, d.f, d.mask, b->bins[i], b->vols[i]));
        SE2N_TRY(fft_half(pl, b->vols[i], true));
        if (p.dynamic) SE2N_TRY(dr_begin(pl, b->dr[i], d.f, d.mask, b->bins[i]));
    }
    SE2N_TRY(batch_interval(b, Tr, true));
    for (int r = 1; r < p.rounds; ++r) {
        for (int i = 0; i < b->count; ++i) {
            if (b->img_fused[i]) continue;
            se2n_plan *pl = b->plan_of[i];
            const se2n_image_desc &d = b->imgs[i];
            SE2N_TRY(fft_half(pl, b->vols[i], false));
            SE2N_TRY(restore_impl(pl, p.dynamic ? &b->dr[i] : nullptr, b->vols[i], d.f, d.mask, b->bins[i],
                                  (float)(1.0 / (double)pl->HW), (float)p.eps, (float)p.guard, true));
            SE2N_TRY(fft_half(pl, b->vols[i], true));
        }
        SE2N_TRY(batch_interval(b, Tr, true));
    }
    for (int i = 0; i < b->count; ++i) {
        if (b->img_fused[i]) continue;
        se2n_plan *pl = b->plan_of[i];
        const se2n_image_desc &d = b->imgs[i];
        const float inv_hw = (float)(1.0 / (double)pl->HW);
        SE2N_TRY(fft_half(pl, b->vols[i], false));
        float scale = inv_hw;
        if (p.final_mix) {
            SE2N_TRY(restore_impl(pl, p.dynamic ? &b->dr[i] : nullptr, b->vols[i], d.f, d.mask, b->bins[i], inv_hw,
                                  (float)p.eps, (float)p.guard, true));
            scale = 1.0f;
        }
        SE2N_TRY(project_half_impl(pl, b->vols[i], scale, p.proj, p.reinject ? d.f : nullptr,
                                   p.reinject ? d.mask : nullptr, d.out));
    }
    // the images on the row and column passes, each whole inpaint in turn
    // (images of one shape share their plan's buffers and propagators)
    for (int i = 0; i < b->count; ++i) {
        if (!b->img_fused[i]) continue;
        se2n_params q = p;
        q.N = b->imgs[i].N;
        SE2N_TRY(inpaint_impl(b->plan_of[i], b->imgs[i].f, b->imgs[i].mask, b->bins[i], &q, b->vols[i],
                              b->imgs[i].out, true));
    }
    return SE2N_OK;
}

// With every image on propagators, the images of one shape touch only that
// shape's plan (its buffers, transforms and propagators) and their own
// volumes, so the shapes are independent: each runs its images in turn (the
// sequence se2n_inpaint enqueues for one image) on a stream of its own,
// forked from the batch's stream and joined back to it, and the graph holds
// the shapes side by side where one stream would run every kernel of every
// image one after another.
bool batch_by_shape(const se2n_batch *b) {
    return !b->p.full_spectrum && b->prop_images == b->count && b->plans.size() > 1;
}

se2n_status enqueue_by_shape(se2n_batch *b, const std::vector<cudaStream_t> &ss, const std::vector<cudaEvent_t> &evs,
                             cudaEvent_t fork) {
    if (cudaEventRecord(fork, b->stream) != cudaSuccess) return SE2N_ECUDA;
    se2n_status st = SE2N_OK;
    size_t forked = 0;
    for (; forked < b->plans.size() && st == SE2N_OK; ++forked) {
        if (cudaStreamWaitEvent(ss[forked], fork, 0) != cudaSuccess) st = SE2N_ECUDA;
        if (st == SE2N_OK) st = se2n_plan_set_stream(b->plans[forked], ss[forked]);
    }
    for (int i = 0; i < b->count && st == SE2N_OK; ++i) {
        se2n_params q = b->p;
        q.N = b->imgs[i].N;
        st = inpaint_impl(b->plan_of[i], b->imgs[i].f, b->imgs[i].mask, b->imgs[i].bins, &q, b->vols[i],
                          b->imgs[i].out, b->img_fused[i]);
    }
    // every forked stream joins back, also after an error, so that the capture ends
    for (size_t k = 0; k < forked; ++k) {
        if (cudaEventRecord(evs[k], ss[k]) != cudaSuccess || cudaStreamWaitEvent(b->stream, evs[k], 0) != cudaSuccess)
            st = SE2N_ECUDA;
        if (se2n_plan_set_stream(b->plans[k], b->stream) != SE2N_OK && st == SE2N_OK) st = SE2N_ECUFFT;
    }
    return st;
}

se2n_status enqueue_batch(se2n_batch *b) {
    const se2n_params &p = b->p;
    if (!p.full_spectrum) return enqueue_batch_half(b);
    const double Tr = p.T / p.rounds;
    for (int i = 0; i < b->count; ++i) {
        se2n_plan *pl = b->plan_of[i];
        const se2n_image_desc &d = b->imgs[i];
        if (d.bins) {
            if (cudaMemcpyAsync(b->bins[i], d.bins, (size_t)pl->HW, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
                return SE2N_ECUDA;
        } else {
            SE2N_TRY(orient_impl(pl, d.f, d.mask, p.sigma_smooth, p.flat_tol, b->bins[i]));
        }
        SE2N_TRY(lift_impl(pl, d.f, d.mask, b->bins[i], b->vols[i]));
        SE2N_TRY(fft(pl, pl->fft_vol, b->vols[i], CUFFT_FORWARD));
        if (p.dynamic) SE2N_TRY(dr_begin(pl, b->dr[i], d.f, d.mask, b->bins[i]));
    }
    SE2N_TRY(batch_interval(b, Tr, false));
    for (int r = 1; r < p.rounds; ++r) {
        for (int i = 0; i < b->count; ++i) {
            se2n_plan *pl = b->plan_of[i];
            const se2n_image_desc &d = b->imgs[i];
            SE2N_TRY(fft(pl, pl->fft_vol, b->vols[i], CUFFT_INVERSE));
            SE2N_TRY(restore_impl(pl, p.dynamic ? &b->dr[i] : nullptr, b->vols[i], d.f, d.mask, b->bins[i],
                                  (float)(1.0 / (double)pl->HW), (float)p.eps, (float)p.guard, false));
            SE2N_TRY(fft(pl, pl->fft_vol, b->vols[i], CUFFT_FORWARD));
        }
        SE2N_TRY(batch_interval(b, Tr, false));
    }
    for (int i = 0; i < b->count; ++i) {
        se2n_plan *pl = b->plan_of[i];
        const se2n_image_desc &d = b->imgs[i];
        const float inv_hw = (float)(1.0 / (double)pl->HW);
        SE2N_TRY(fft(pl, pl->fft_vol, b->vols[i], CUFFT_INVERSE));
        float scale = inv_hw;
        if (p.final_mix) {
            SE2N_TRY(restore_impl(pl, p.dynamic ? &b->dr[i] : nullptr, b->vols[i], d.f, d.mask, b->bins[i], inv_hw,
                                  (float)p.eps, (float)p.guard, false));
            scale = 1.0f;
        }
        SE2N_TRY(project_impl(pl, b->vols[i], scale, p.proj, p.reinject ? d.f : nullptr,
                              p.reinject ? d.mask : nullptr, d.out));
    }
    return SE2N_OK;
}

void free_batch(se2n_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (DrState &d : b->dr) dr_free(d);
    for (se2n_plan *pl : b->plans) {
        cudaStreamSynchronize(pl->stream);
        free_plan(pl);
    }
    cudaFree(b->arena);
    cudaFree(b->d_tables);
    cudaFree(b->d_imgs);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

se2n_status create_batch(se2n_batch *b, const se2n_image_desc *imgs) {
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return SE2N_ECUDA;
    b->imgs.assign(imgs, imgs + b->count);
    // plans per distinct shape
    b->plan_of.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        const se2n_image_desc &d = imgs[i];
        se2n_plan *found = nullptr;
        for (se2n_plan *pl : b->plans)
            if (pl->H == d.H && pl->W == d.W && pl->N == d.N) found = pl;
        if (!found) {
            SE2N_TRY(se2n_plan_create(&found, d.H, d.W, d.N, b->angle_conv, (void *)b->stream));
            b->plans.push_back(found);
        }
        b->plan_of[i] = found;
        b->updates += (double)d.H * d.W * d.N * b->p.steps * b->p.rounds;
    }
    // one arena: every volume 256-byte aligned, then the bin maps
    std::vector<size_t> voff(b->count), boff(b->count);
    size_t off = 0;
    for (int i = 0; i < b->count; ++i) {
        voff[i] = off;
        off += ((size_t)imgs[i].H * imgs[i].W * imgs[i].N * sizeof(float2) + 255) / 256 * 256;
    }
    b->vol_bytes = off;
    for (int i = 0; i < b->count; ++i) {
        boff[i] = off;
        off += ((size_t)imgs[i].H * imgs[i].W + 255) / 256 * 256;
    }
    e = cudaMalloc(&b->arena, off);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
    b->vols.resize(b->count);
    b->bins.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        b->vols[i] = (float2 *)(b->arena + voff[i]);
        b->bins[i] = (uint8_t *)(b->arena + boff[i]);
    }
    if (b->p.dynamic) {
        b->dr.resize(b->count);
        for (int i = 0; i < b->count; ++i) SE2N_TRY(dr_alloc(b->dr[i], (long long)imgs[i].H * imgs[i].W));
    }
    // angle tables, one per distinct N, cos[N] then sin[N]
    std::vector<float> tables;
    std::vector<int> table_N, table_off;
    b->h_imgs.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        const int N = imgs[i].N;
        int t = -1;
        for (size_t j = 0; j < table_N.size(); ++j)
            if (table_N[j] == N) t = table_off[j];
        if (t < 0) {
            t = (int)tables.size();
            table_N.push_back(N);
            table_off.push_back(t);
            std::vector<float> cs(N), sn(N);
            angle_table(N, b->angle_conv, cs.data(), sn.data(), N);
            tables.insert(tables.end(), cs.begin(), cs.end());
            tables.insert(tables.end(), sn.begin(), sn.end());
        }
        BatchImage &bi = b->h_imgs[i];
        bi.vol = b->vols[i];
        bi.H = imgs[i].H;
        bi.W = imgs[i].W;
        bi.Wc = b->p.full_spectrum ? bi.W : bi.W / 2 + 1;
        bi.HW = (long long)bi.H * bi.Wc;
        bi.N = N;
        bi.table = t;
    }
    e = cudaMalloc(&b->d_tables, sizeof(float) * tables.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_imgs, sizeof(BatchImage) * b->count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 256);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_tables, tables.data(), sizeof(float) * tables.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_imgs, b->h_imgs.data(), sizeof(BatchImage) * b->count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
    // numerical path (as se2n_diffuse chooses it for one interval)
    const double Tr = b->p.T / b->p.rounds;
    const double bdt = b->p.beta * Tr / b->p.steps;
    b->split = (b->p.diffuse_flags & SE2N_DIFFUSE_SPLIT_DIAG) || b->p.beta * Tr > 8.0;
    b->fast = !(b->p.diffuse_flags & SE2N_DIFFUSE_FULL_CORRECTION) && se2n_diffuse_truncation_ok(bdt);
    if (cudaMemsetAsync(b->arena, 0, b->vol_bytes, b->stream) != cudaSuccess) return SE2N_ECUDA;
    // transforms of the Hermitian-half path are planned before the capture
    if (!b->p.full_spectrum)
        for (se2n_plan *pl : b->plans) SE2N_TRY(ensure_half(pl));
    // so is the propagators' memory; the graph builds them (once per shape)
    choose_propagators(b);
    for (se2n_plan *pl : b->plans) {
        bool used = false;
        for (int i = 0; i < b->count; ++i) used = used || (b->img_prop[i] && b->plan_of[i] == pl);
        if (!used) continue;
        bool fused = false;
        for (int i = 0; i < b->count; ++i) fused = fused || (b->img_fused[i] && b->plan_of[i] == pl);
        if (fused) {
            // everything the whole inpaints allocate or create, before the capture
            SE2N_TRY(col_ensure(pl));
            SE2N_TRY(side_ensure(pl));
            SE2N_TRY(prop_reserve(pl, true, PROP_CHUNKS));
            if (b->p.dynamic) SE2N_TRY(dr_alloc(pl->dr, pl->HW));
        } else {
            SE2N_TRY(prop_reserve(pl, !b->p.full_spectrum, se2n_prop_apply_fmt(pl->N, !b->p.full_spectrum)));
        }
        if (se2n_prop_prepare(pl->N) != cudaSuccess) return SE2N_ECUDA;
        pl->prop_valid = false;
    }
    if (b->flags_autotune) {
        SE2N_TRY(autotune(b));
    } else {
        SE2N_TRY(set_shape(b, 0, 8, 256));
    }
    // capture the whole method into a graph: the shapes side by side when
    // they are independent (their streams and events exist for the capture only)
    const bool by_shape = batch_by_shape(b);
    std::vector<cudaStream_t> ss;
    std::vector<cudaEvent_t> evs;
    cudaEvent_t fork = nullptr;
    auto release = [&]() {
        for (cudaStream_t x : ss) cudaStreamDestroy(x);
        for (cudaEvent_t x : evs) cudaEventDestroy(x);
        if (fork) cudaEventDestroy(fork);
    };
    if (by_shape) {
        if (b->p.dynamic)
            for (se2n_plan *pl : b->plans) SE2N_TRY(dr_alloc(pl->dr, pl->HW));
        bool ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
        for (size_t k = 0; k < b->plans.size() && ok; ++k) {
            cudaStream_t x = nullptr;
            cudaEvent_t e = nullptr;
            ok = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) ss.push_back(x);
            ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
            if (ok) evs.push_back(e);
        }
        if (!ok) {
            release();
            return SE2N_ECUDA;
        }
    }
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        release();
        return SE2N_ECUDA;
    }
    se2n_status st = by_shape ? enqueue_by_shape(b, ss, evs, fork) : enqueue_batch(b);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    release();
    if (st != SE2N_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return SE2N_ECUDA;
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return SE2N_ECUDA;
    return SE2N_OK;
}

}  // namespace

extern "C" {

se2n_status se2n_batch_create(se2n_batch **out, const se2n_image_desc *imgs, int count, const se2n_params *p,
                              int angle_conv, int flags, void *stream) {
    if (!out || !imgs || count < 1 || !p || (angle_conv != 0 && angle_conv != 1)) return SE2N_EINVAL;
    if (flags & ~SE2N_BATCH_AUTOTUNE) return SE2N_EINVAL;
    for (int i = 0; i < count; ++i) {
        const se2n_image_desc &d = imgs[i];
        if (d.H < 2 || d.W < 2 || (d.H % 2) || (d.W % 2) || (long long)d.H * d.W > (1LL << 28)) return SE2N_EINVAL;
        if (d.N != 16 && d.N != 32 && d.N != 64) return SE2N_EUNSUPPORTED;
        if (!device_ptr(d.f, 8) || !device_ptr(d.mask, 2) || !device_ptr(d.out, 8)) return SE2N_EINVAL;
        if (d.bins && !device_ptr(d.bins, 2)) return SE2N_EINVAL;
    }
    se2n_batch *b = new (std::nothrow) se2n_batch();
    if (!b) return SE2N_ENOMEM;
    b->count = count;
    b->angle_conv = angle_conv;
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        // Graphs cannot be captured on the legacy default stream. A blocking
        // stream of our own is still ordered with the caller's legacy-stream
        // work in both directions.
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault) != cudaSuccess) {
            delete b;
            return SE2N_ECUDA;
        }
        b->own_stream = true;
    }
    b->p = *p;
    b->flags_autotune = (flags & SE2N_BATCH_AUTOTUNE) != 0;
    se2n_status st = SE2N_OK;
    for (int i = 0; i < count && st == SE2N_OK; ++i) {
        se2n_plan probe{};
        probe.N = imgs[i].N;
        se2n_params q = *p;
        q.N = imgs[i].N;
        st = check_params(&probe, &q);
    }
    if (st == SE2N_OK) st = create_batch(b, imgs);
    if (st == SE2N_OK) st = cudaStreamSynchronize(b->stream) == cudaSuccess ? SE2N_OK : SE2N_ECUDA;
    if (st != SE2N_OK) {
        (void)cudaGetLastError();
        free_batch(b);
        return st;
    }
    *out = b;
    return SE2N_OK;
}

se2n_status se2n_batch_run(se2n_batch *b) {
    if (!b) return SE2N_EINVAL;
    return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? SE2N_OK : SE2N_ECUDA;
}

se2n_status se2n_batch_run_per_image(se2n_batch *b) {
    if (!b) return SE2N_EINVAL;
    // the same work as the graph: every shape's propagators built again
    for (se2n_plan *pl : b->plans) pl->prop_valid = false;
    for (int i = 0; i < b->count; ++i) {
        se2n_params q = b->p;
        q.N = b->imgs[i].N;
        // the same integration the batch chose for this image's shape
        if (b->img_prop.empty() || !b->img_prop[i]) q.diffuse_flags &= ~SE2N_DIFFUSE_PROPAGATOR;
        const bool fused = !b->img_fused.empty() && b->img_fused[i];
        SE2N_TRY(inpaint_impl(b->plan_of[i], b->imgs[i].f, b->imgs[i].mask, b->imgs[i].bins, &q, b->vols[i],
                              b->imgs[i].out, fused));
    }
    return SE2N_OK;
}

se2n_status se2n_batch_run_diffusion(se2n_batch *b) {
    if (!b) return SE2N_EINVAL;
    return batch_diffuse(b, b->p.steps, b->p.T / b->p.rounds);
}

se2n_status se2n_batch_get_info(se2n_batch *b, se2n_batch_info *out) {
    if (!b || !out) return SE2N_EINVAL;
    out->images = b->count;
    out->items = b->n_items;
    out->tile_passes = b->passes;
    out->block = b->block;
    out->blocks = b->blocks;
    out->p16 = se2n_batch_config_P(b->config, 16);
    out->p32 = se2n_batch_config_P(b->config, 32);
    out->p64 = se2n_batch_config_P(b->config, 64);
    out->fast = b->fast;
    out->split = b->split;
    out->candidates = b->candidates;
    out->best_ms = b->best_ms;
    out->worst_ms = b->worst_ms;
    out->updates_per_run = b->updates;
    out->volume_bytes = (double)b->vol_bytes;
    out->prop_images = b->prop_images;
    out->fused_images = b->fused_images;
    out->step_updates = 0.0;
    for (int i = 0; i < b->count; ++i)
        if (b->img_prop.empty() || !b->img_prop[i])
            out->step_updates += (double)b->h_imgs[i].HW * b->imgs[i].N * b->p.steps;
    return SE2N_OK;
}

se2n_status se2n_batch_destroy(se2n_batch *b) {
    if (!b) return SE2N_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return SE2N_OK;
}

}  // extern "C"
