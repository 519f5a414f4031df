// The surrogate network object: a 4-level U-Net with 32-64-128-256 channels,
// BF16 weights and activations, FP32 accumulation, trained by its own
// forward and backward kernels (nn.cu) with Adam on FP32 master weights.
//
// Layers (3x3 convolutions with ReLU unless noted), H x W input:
//   enc0a 8->32, enc0b 32->32                      (H x W)       -> e0
//   pool, enc1a 32->64, enc1b 64->64                (H/2)         -> e1
//   pool, enc2a 64->128, enc2b 128->128             (H/4)         -> e2
//   pool, enc3a 128->256, enc3b 256->256            (H/8)         -> e3
//   dec2a [up(e3), e2] 384->128, dec2b 128->128     (H/4)         -> d2
//   dec1a [up(d2), e1] 192->64, dec1b 64->64        (H/2)         -> d1
//   dec0a [up(d1), e0] 96->32, dec0b 32->32         (H)           -> d0
//   head: 1x1 32->1, no activation                                -> out
// Input channels: f (zero on corrupted pixels), the mask, 6 zero channels.
// Pooling is 2x2 average, upsampling nearest; "up" and the concatenation
// are read on the fly by the decoder convolutions.
//
// Parameters, one flat FP32 vector: for each conv layer in the order above
// W[cout][9][cin] (tap = (dy+1)*3 + (dx+1)) then b[cout]; then the head
// w[32], b[1].
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "nn.h"
#include "se2n_internal.h"

namespace {

struct LayerSpec {
    int cin, cout, level;
    int lo_ch;  // channels read upsampled from the level below (decoder first convs), else 0
};

const LayerSpec kLayers[14] = {
    {8, 32, 0, 0},     {32, 32, 0, 0},    {32, 64, 1, 0},   {64, 64, 1, 0},   {64, 128, 2, 0},
    {128, 128, 2, 0},  {128, 256, 3, 0},  {256, 256, 3, 0}, {384, 128, 2, 256}, {128, 128, 2, 0},
    {192, 64, 1, 128}, {64, 64, 1, 0},    {96, 32, 0, 64},  {32, 32, 0, 0},
};

}  // namespace

struct se2n_unet {
    int B = 0, H = 0, W = 0;
    cudaStream_t stream = nullptr;
    long long n_params = 0;
    size_t w_off[14], b_off[14], hw_off = 0, hb_off = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pb = nullptr;
    int step = 0;
    // activations and their gradients (bf16), one arena
    __nv_bfloat16 *arena = nullptr;
    __nv_bfloat16 *x0, *a[4], *e[4], *pl[4], *c[3], *d[3];
    __nv_bfloat16 *gd[3], *gc[3], *gup[3], *gskip[3], *ge[4], *ga[4], *gp[4];
    __nv_bfloat16 *cat[3];  // decoder inputs [up(below), skip]; e[0..2] live inside them
    int e_ld[4];            // channels per pixel of the tensor e[l] lives in
    float *out = nullptr, *target = nullptr, *loss = nullptr, *resid = nullptr;
    __nv_bfloat16 *wt = nullptr;  // one layer's weights rearranged for the data gradient
};

namespace {

se2n_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return SE2N_OK;
    return e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA;
}

#define TRY(expr)                              \
    do {                                       \
        se2n_status _s = (expr);               \
        if (_s != SE2N_OK) return _s;          \
    } while (0)
#define TRYC(expr) TRY(cuda_st(expr))

// A tensor-core convolution that gave up on a bounded wait (never expected)
// is reported by the next synchronous call as SE2N_ECUDA.
se2n_status check_tc() {
    int f = 0;
    TRYC(se2n::nn::tc_fault(&f, true));
    return f ? SE2N_ECUDA : SE2N_OK;
}

long long level_pixels(const se2n_unet *u, int count, int level) {
    return (long long)count * (u->H >> level) * (u->W >> level);
}

bool dev_ptr(const void *p, size_t align) {
    if (!p || ((uintptr_t)p % align) != 0) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// keep: write every activation the backward pass reads (the last
// convolution's output d0 is needed only there)
se2n_status forward(se2n_unet *u, const float *f, const uint8_t *mask, int n, bool keep) {
    using namespace se2n::nn;
    cudaStream_t s = u->stream;
    const int H = u->H, W = u->W;
    auto Wt = [&](int l) { return u->pb + u->w_off[l]; };
    auto Bi = [&](int l) { return u->p + u->b_off[l]; };
    for (int l = 0; l < 4; ++l) {
        const int Hl = H >> l, Wl = W >> l;
        const LayerSpec &A = kLayers[2 * l], &Bb = kLayers[2 * l + 1];
        if (l == 0) {
            // the first layer reads the image and mask directly (2 meaningful input channels)
            TRYC(conv0_direct(f, mask, Wt(0), Bi(0), u->a[0], n, H, W, s));
        } else {
            TRYC(pool(u->e[l - 1], u->e_ld[l - 1], u->pl[l], n, H >> (l - 1), W >> (l - 1), kLayers[2 * l - 1].cout, s));
            TRYC(conv_forward(u->pl[l], nullptr, 0, n, Hl, Wl, A.cin, Wt(2 * l), Bi(2 * l), A.cout, 1, u->a[l], A.cout,
                              s));
        }
        // e[l] (l < 3) is written straight into the skip channels of decoder level l's input
        TRYC(conv_forward(u->a[l], nullptr, 0, n, Hl, Wl, Bb.cin, Wt(2 * l + 1), Bi(2 * l + 1), Bb.cout, 1, u->e[l],
                          u->e_ld[l], s));
    }
    // decoder levels 2, 1, 0 (layer indices 8..13)
    const __nv_bfloat16 *below = u->e[3];
    for (int k = 0; k < 3; ++k) {
        const int level = 2 - k;
        const int la = 8 + 2 * k, lb = 9 + 2 * k;
        const LayerSpec &A = kLayers[la], &Bb = kLayers[lb];
        const int Hl = H >> level, Wl = W >> level;
        // the input [up(below), e[level]] is one NHWC tensor (read with TMA boxes):
        // e[level] is already in it, the upsampled half is written here
        TRYC(upsample_into(below, A.lo_ch, u->cat[k], A.cin, n, Hl, Wl, s));
        TRYC(conv_forward(u->cat[k], nullptr, 0, n, Hl, Wl, A.cin, Wt(la), Bi(la), A.cout, 1, u->c[k], A.cout, s));
        if (k == 2) {
            // last convolution with the head and the input skip fused, when the tile shape allows
            const HeadArgs h{u->p + u->hw_off, u->p + u->hb_off, f, mask, u->out};
            const cudaError_t e = conv_forward_tma(u->c[k], n, Hl, Wl, Bb.cin, Wt(lb), Bi(lb), Bb.cout, 1,
                                                   keep ? u->d[k] : nullptr, Bb.cout, &h, s);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotSupported) return cuda_st(e);
        }
        TRYC(conv_forward(u->c[k], nullptr, 0, n, Hl, Wl, Bb.cin, Wt(lb), Bi(lb), Bb.cout, 1, u->d[k], Bb.cout, s));
        below = u->d[k];
        if (k == 2)
            TRYC(head(u->d[2], u->p + u->hw_off, u->p + u->hb_off, f, mask, u->out, (long long)n * H * W, 32, s));
    }
    return SE2N_OK;
}

se2n_status backward(se2n_unet *u, const float *f, const uint8_t *mask, int n) {
    using namespace se2n::nn;
    cudaStream_t s = u->stream;
    const int H = u->H, W = u->W;
    auto Wt = [&](int l) { return u->pb + u->w_off[l]; };
    auto dW = [&](int l) { return u->g + u->w_off[l]; };
    auto dB = [&](int l) { return u->g + u->b_off[l]; };
    // the first layer's input as the weight gradient reads it (8 channels: f m, m, zeros)
    TRYC(pack_input(f, mask, u->x0, (long long)n * H * W, s));
    TRYC(cudaMemsetAsync(u->g, 0, sizeof(float) * u->n_params, s));
    TRYC(cudaMemsetAsync(u->loss, 0, sizeof(float), s));
    TRYC(loss_head_backward(u->out, u->target, u->d[2], u->p + u->hw_off, u->gd[2], u->g + u->hw_off,
                            u->g + u->hb_off, u->loss, (long long)n * H * W, 32, s));
    // decoder, from level 0 up: gradient into d[k] is gd[k]
    for (int k = 2; k >= 0; --k) {
        const int level = 2 - k;
        const int la = 8 + 2 * k, lb = 9 + 2 * k;
        const LayerSpec &A = kLayers[la], &Bb = kLayers[lb];
        const int Hl = H >> level, Wl = W >> level;
        const long long P = level_pixels(u, n, level);
        // second conv: c[k] -> d[k]
        TRYC(conv_backward_weight(u->gd[k], n, Hl, Wl, Bb.cout, u->c[k], nullptr, 0, Bb.cin, dW(lb), s));
        TRYC(colsum(u->gd[k], P, Bb.cout, dB(lb), s));
        TRYC(conv_backward_data(u->gd[k], n, Hl, Wl, Bb.cout, Wt(lb), Bb.cin, u->c[k], u->gc[k], nullptr, Bb.cin, u->wt, s));
        // first conv: [up(below), e[level]] -> c[k]
        TRYC(conv_backward_weight(u->gc[k], n, Hl, Wl, A.cout, u->cat[k], nullptr, 0, A.cin, dW(la), s));
        TRYC(colsum(u->gc[k], P, A.cout, dB(la), s));
        TRYC(conv_backward_data(u->gc[k], n, Hl, Wl, A.cout, Wt(la), A.cin, nullptr, u->gup[k], u->gskip[k],
                                A.lo_ch, u->wt, s));
        // gradient into the tensor below (half resolution), through the upsampling
        if (k > 0) {
            TRYC(up_backward_mask(u->gup[k], u->d[k - 1], u->gd[k - 1], n, Hl / 2, Wl / 2, A.lo_ch, s));
        } else {
            TRYC(up_backward_mask(u->gup[k], u->e[3], u->ge[3], n, Hl / 2, Wl / 2, A.lo_ch, s));
        }
    }
    // encoder, from the bottleneck down: gradient into e[l] is ge[l]
    for (int l = 3; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l;
        const long long P = level_pixels(u, n, l);
        const LayerSpec &A = kLayers[2 * l], &Bb = kLayers[2 * l + 1];
        if (l < 3) {
            // e[l] feeds the pool of level l+1 (gradient gp[l+1]) and the skip of decoder level l
            TRYC(pool_backward_add_mask(u->gp[l + 1], u->gskip[2 - l], u->e[l], u->e_ld[l], u->ge[l], n, Hl, Wl,
                                        Bb.cout, s));
        }
        const __nv_bfloat16 *in = (l == 0) ? u->x0 : u->pl[l];
        TRYC(conv_backward_weight(u->ge[l], n, Hl, Wl, Bb.cout, u->a[l], nullptr, 0, Bb.cin, dW(2 * l + 1), s));
        TRYC(colsum(u->ge[l], P, Bb.cout, dB(2 * l + 1), s));
        TRYC(conv_backward_data(u->ge[l], n, Hl, Wl, Bb.cout, Wt(2 * l + 1), Bb.cin, u->a[l], u->ga[l], nullptr,
                                Bb.cin, u->wt, s));
        TRYC(conv_backward_weight(u->ga[l], n, Hl, Wl, A.cout, in, nullptr, 0, A.cin, dW(2 * l), s));
        TRYC(colsum(u->ga[l], P, A.cout, dB(2 * l), s));
        if (l > 0) {
            TRYC(conv_backward_data(u->ga[l], n, Hl, Wl, A.cout, Wt(2 * l), A.cin, nullptr, u->gp[l], nullptr, A.cin, u->wt, s));
        }
    }
    return SE2N_OK;
}

// Deterministic He-normal initialisation (splitmix64 + Box-Muller), host side.
uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit(uint64_t &x) { return ((splitmix(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

}  // namespace

extern "C" {

se2n_status se2n_unet_create(se2n_unet **out, int batch, int H, int W, void *stream) {
    if (!out || batch < 1 || H < 8 || W < 8 || (H % 8) || (W % 8)) return SE2N_EINVAL;
    if ((long long)batch * H * W > (1LL << 30)) return SE2N_EINVAL;
    se2n_unet *u = new (std::nothrow) se2n_unet();
    if (!u) return SE2N_ENOMEM;
    u->B = batch;
    u->H = H;
    u->W = W;
    u->stream = (cudaStream_t)stream;
    size_t off = 0;
    for (int l = 0; l < 14; ++l) {
        u->w_off[l] = off;
        off += (size_t)kLayers[l].cout * 9 * kLayers[l].cin;
        u->b_off[l] = off;
        off += kLayers[l].cout;
    }
    u->hw_off = off;
    off += 32;
    u->hb_off = off;
    off += 1;
    u->n_params = (long long)off;
    // activation arena sizes (elements)
    const long long P0 = (long long)batch * H * W;
    auto P = [&](int l) { return P0 >> (2 * l); };
    std::vector<std::pair<__nv_bfloat16 **, long long>> bufs;
    bufs.push_back({&u->x0, P(0) * 8});
    for (int l = 0; l < 4; ++l) {
        bufs.push_back({&u->a[l], P(l) * kLayers[2 * l].cout});
        if (l == 3) bufs.push_back({&u->e[l], P(l) * kLayers[2 * l + 1].cout});
        bufs.push_back({&u->ga[l], P(l) * kLayers[2 * l].cout});
        bufs.push_back({&u->ge[l], P(l) * kLayers[2 * l + 1].cout});
        bufs.push_back({&u->pl[l], l > 0 ? P(l) * kLayers[2 * l - 1].cout : 8});
        bufs.push_back({&u->gp[l], l > 0 ? P(l) * kLayers[2 * l - 1].cout : 8});
    }
    for (int k = 0; k < 3; ++k) {
        const int level = 2 - k;
        const LayerSpec &A = kLayers[8 + 2 * k];
        bufs.push_back({&u->c[k], P(level) * A.cout});
        bufs.push_back({&u->d[k], P(level) * A.cout});
        bufs.push_back({&u->gc[k], P(level) * A.cout});
        bufs.push_back({&u->gd[k], P(level) * A.cout});
        bufs.push_back({&u->gup[k], P(level) * A.lo_ch});
        bufs.push_back({&u->gskip[k], P(level) * (A.cin - A.lo_ch)});
        bufs.push_back({&u->cat[k], P(level) * A.cin});
    }
    long long total = 0;
    for (auto &b : bufs) total += (b.second + 127) / 128 * 128;
    cudaError_t e = cudaMalloc(&u->arena, sizeof(__nv_bfloat16) * total);
    long long o = 0;
    if (e == cudaSuccess)
        for (auto &b : bufs) {
            *b.first = u->arena + o;
            o += (b.second + 127) / 128 * 128;
        }
    // e[l], l < 3: the skip channels of decoder level l's input (after the upsampled ones)
    for (int l = 0; l < 4; ++l) u->e_ld[l] = kLayers[2 * l + 1].cout;
    if (e == cudaSuccess)
        for (int l = 0; l < 3; ++l) {
            const LayerSpec &D = kLayers[8 + 2 * (2 - l)];
            u->e[l] = u->cat[2 - l] + D.lo_ch;
            u->e_ld[l] = D.cin;
        }
    const size_t np = (size_t)u->n_params;
    if (e == cudaSuccess) e = cudaMalloc(&u->p, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&u->g, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&u->m, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&u->v, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&u->pb, sizeof(__nv_bfloat16) * np);
    if (e == cudaSuccess) e = cudaMalloc(&u->out, sizeof(float) * P0);
    if (e == cudaSuccess) e = cudaMalloc(&u->target, sizeof(float) * P0);
    if (e == cudaSuccess) e = cudaMalloc(&u->loss, 256);
    if (e == cudaSuccess) e = cudaMalloc(&u->resid, sizeof(float) * batch);
    size_t wmax = 0;
    for (int l = 0; l < 14; ++l) {
        const size_t nw = (size_t)kLayers[l].cout * 9 * kLayers[l].cin;
        if (nw > wmax) wmax = nw;
    }
    if (e == cudaSuccess) e = cudaMalloc(&u->wt, sizeof(__nv_bfloat16) * wmax);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->p, 0, sizeof(float) * np, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, sizeof(float) * np, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, sizeof(float) * np, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->pb, 0, sizeof(__nv_bfloat16) * np, u->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) {
        cudaFree(u->arena);
        cudaFree(u->p);
        cudaFree(u->g);
        cudaFree(u->m);
        cudaFree(u->v);
        cudaFree(u->pb);
        cudaFree(u->out);
        cudaFree(u->target);
        cudaFree(u->loss);
        cudaFree(u->resid);
        cudaFree(u->wt);
        delete u;
        return cuda_st(e);
    }
    *out = u;
    return SE2N_OK;
}

se2n_status se2n_unet_destroy(se2n_unet *u) {
    if (!u) return SE2N_OK;
    cudaStreamSynchronize(u->stream);
    cudaFree(u->arena);
    cudaFree(u->p);
    cudaFree(u->g);
    cudaFree(u->m);
    cudaFree(u->v);
    cudaFree(u->pb);
    cudaFree(u->out);
    cudaFree(u->target);
    cudaFree(u->loss);
    cudaFree(u->resid);
    cudaFree(u->wt);
    delete u;
    return SE2N_OK;
}

se2n_status se2n_unet_param_count(const se2n_unet *u, long long *n) {
    if (!u || !n) return SE2N_EINVAL;
    *n = u->n_params;
    return SE2N_OK;
}

se2n_status se2n_unet_set_params(se2n_unet *u, const float *host) {
    if (!u || !host) return SE2N_EINVAL;
    TRYC(cudaMemcpyAsync(u->p, host, sizeof(float) * u->n_params, cudaMemcpyHostToDevice, u->stream));
    TRYC(se2n::nn::to_bf16(u->p, u->pb, u->n_params, u->stream));
    TRYC(cudaMemsetAsync(u->m, 0, sizeof(float) * u->n_params, u->stream));
    TRYC(cudaMemsetAsync(u->v, 0, sizeof(float) * u->n_params, u->stream));
    u->step = 0;
    return cuda_st(cudaStreamSynchronize(u->stream));
}

se2n_status se2n_unet_get_params(se2n_unet *u, float *host) {
    if (!u || !host) return SE2N_EINVAL;
    TRYC(cudaMemcpyAsync(host, u->p, sizeof(float) * u->n_params, cudaMemcpyDeviceToHost, u->stream));
    TRYC(cudaStreamSynchronize(u->stream));
    return check_tc();
}

se2n_status se2n_unet_get_grads(se2n_unet *u, float *host) {
    if (!u || !host) return SE2N_EINVAL;
    TRYC(cudaMemcpyAsync(host, u->g, sizeof(float) * u->n_params, cudaMemcpyDeviceToHost, u->stream));
    TRYC(cudaStreamSynchronize(u->stream));
    return check_tc();
}

se2n_status se2n_unet_init(se2n_unet *u, unsigned long long seed) {
    if (!u) return SE2N_EINVAL;
    std::vector<float> h((size_t)u->n_params, 0.0f);
    uint64_t st = seed;
    for (int l = 0; l < 14; ++l) {
        const int fan_in = 9 * (l == 0 ? 2 : kLayers[l].cin);  // the input has 2 meaningful channels
        const double sd = sqrt(2.0 / fan_in);
        const size_t n = (size_t)kLayers[l].cout * 9 * kLayers[l].cin;
        for (size_t i = 0; i < n; ++i) {
            const double u1 = unit(st), u2 = unit(st);
            h[u->w_off[l] + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
        }
    }
    // the head starts at zero: the untrained network is the identity on the
    // masked input (out = f on known pixels, 0 elsewhere), and training
    // grows the correction from there
    return se2n_unet_set_params(u, h.data());
}

se2n_status se2n_unet_forward(se2n_unet *u, const float *f, const uint8_t *mask, int count, float *out) {
    if (!u || count < 1 || count > u->B) return SE2N_EINVAL;
    if (!dev_ptr(f, 4) || !dev_ptr(mask, 1) || !dev_ptr(out, 4)) return SE2N_EINVAL;
    TRY(forward(u, f, mask, count, false));
    return cuda_st(cudaMemcpyAsync(out, u->out, sizeof(float) * count * u->H * u->W, cudaMemcpyDeviceToDevice,
                                   u->stream));
}

se2n_status se2n_unet_backward(se2n_unet *u, const float *f, const uint8_t *mask, const float *target, int count,
                               float *loss_device) {
    if (!u || count < 1 || count > u->B) return SE2N_EINVAL;
    if (!dev_ptr(f, 4) || !dev_ptr(mask, 1) || !dev_ptr(target, 4)) return SE2N_EINVAL;
    if (loss_device && !dev_ptr(loss_device, 4)) return SE2N_EINVAL;
    TRYC(cudaMemcpyAsync(u->target, target, sizeof(float) * count * u->H * u->W, cudaMemcpyDeviceToDevice,
                         u->stream));
    TRY(forward(u, f, mask, count, true));
    TRY(backward(u, f, mask, count));
    if (loss_device) TRYC(cudaMemcpyAsync(loss_device, u->loss, sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
    return SE2N_OK;
}

se2n_status se2n_unet_adam(se2n_unet *u, double lr, double beta1, double beta2, double eps) {
    if (!u || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return SE2N_EINVAL;
    u->step += 1;
    return cuda_st(se2n::nn::adam(u->p, u->g, u->m, u->v, u->pb, u->n_params, (float)lr, (float)beta1, (float)beta2,
                                  (float)eps, u->step, u->stream));
}

se2n_status se2n_unet_train_step(se2n_unet *u, const float *f, const uint8_t *mask, const float *target, int count,
                                 double lr, float *loss_device) {
    TRY(se2n_unet_backward(u, f, mask, target, count, loss_device));
    return se2n_unet_adam(u, lr, 0.9, 0.999, 1e-8);
}

se2n_status se2n_surrogate_inpaint(se2n_unet *u, se2n_plan *plan, const se2n_params *p, const float *f,
                                   const uint8_t *mask, int count, double threshold, void *vol_scratch, float *out,
                                   float *residual_host, int *fallbacks) {
    if (!u || !plan || !p || count < 1 || count > u->B || !(threshold >= 0.0)) return SE2N_EINVAL;
    if (plan->H != u->H || plan->W != u->W) return SE2N_EINVAL;
    TRY(se2n_unet_forward(u, f, mask, count, out));
    const int HW = u->H * u->W;
    TRYC(se2n::nn::known_residual(out, f, mask, count, HW, u->resid, u->stream));
    std::vector<float> r(count);
    TRYC(cudaMemcpyAsync(r.data(), u->resid, sizeof(float) * count, cudaMemcpyDeviceToHost, u->stream));
    TRYC(cudaStreamSynchronize(u->stream));
    TRY(check_tc());
    int nf = 0;
    for (int i = 0; i < count; ++i) {
        if (residual_host) residual_host[i] = r[i];
        if (r[i] > threshold) {
            // the method itself for the images the network does not fit
            TRY(se2n_inpaint(plan, f + (long long)i * HW, mask + (long long)i * HW, nullptr, p, vol_scratch,
                             out + (long long)i * HW));
            ++nf;
        }
    }
    if (fallbacks) *fallbacks = nf;
    return SE2N_OK;
}

}  // extern "C"
