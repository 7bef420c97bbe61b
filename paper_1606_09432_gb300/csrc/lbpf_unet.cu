// The learned surrogate's network runtime: a 2D U-Net of `levels` levels
// with base * 2^l channels at level l (default 3 levels, base 16: 16, 32, 64
// channels), two periodic 3x3 convolutions + ReLU per level on the way down
// (2x2 average pooling between levels) and on the way up (nearest 2x
// upsampling concatenated with the level's skip), and a 1x1 head.
// Input per site: (phi, u, cos 4 theta, sin 4 theta, eps) zero-padded to 16
// channels; output: (d phi, d u), the change of phi and u over the jump, the
// phi channel gated by (1 - phi^2) so that the bulk phases stay untouched.
// Forward, hand-written backward and Adam run in the kernels of lbpf_nn.cu
// (3x3 convolutions and their weight gradients on the tensor cores).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbpf.h"
#include "lbpf_nn.cuh"

using namespace lbpf_nn;

namespace {

constexpr int kIn = 5;      // input channels before padding
constexpr int kInPad = 16;  // padded input channels
constexpr int kOut = 2;

struct Conv {
    int cin, cout;
    long long off_w, off_b;  // offsets in the flat FP32 parameter vector
    __nv_bfloat16* wb = nullptr;   // BF16 copy [tap][cout][cin]
    __nv_bfloat16* wt = nullptr;   // flipped BF16 weights for the data gradient
};

}  // namespace

struct lbpf_net {
    int H = 0, W = 0, N = 0, levels = 3, base = 16;
    cudaStream_t stream = nullptr;
    std::vector<Conv> conv;  // 4 levels - 2 3x3 convolutions: encoder level by level, then decoder top-down
    long long off_hw = 0, off_hb = 0, n_params = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 params, grads, Adam moments
    __nv_bfloat16* pb = nullptr;  // BF16 copies of the 3x3 weights and their flipped forms
    int adam_t = 0;
    float loss_alpha = 0.f;  // interface weight of the training loss
    // activations (N, H >> l, W >> l, c) per level l: encoder convolution
    // outputs ea, e; pooled input pl (l >= 1); decoder concatenation u and
    // outputs da, d (l < levels - 1)
    float *xin = nullptr, *out = nullptr;
    std::vector<float*> ea, e, pl, u, da, d;
    // gradient scratch per level (two of the level's widest channel count)
    // and the skip gradients of the decoder levels
    std::vector<float*> ga, gb, gskip;
    float* g_out = nullptr;
    double* d_loss = nullptr;
    std::vector<void*> allocs;
    std::string err;

    int ch(int l) const { return base << l; }
    float* top() const { return levels > 1 ? d[0] : e[0]; }
};

namespace {

thread_local std::string t_net_err;

int net_fail(lbpf_net* n, int code, const char* msg)
{
    if (n)
        n->err = msg;
    else
        t_net_err = msg;
    return code;
}

#define NK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return net_fail(net, LBPF_ECUDA, cudaGetErrorString(e_));               \
    } while (0)

float* alloc_f(lbpf_net* net, long long n)
{
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(float) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    net->allocs.push_back(p);
    cudaMemsetAsync(p, 0, sizeof(float) * (size_t)(n > 0 ? n : 1), net->stream);
    return static_cast<float*>(p);
}

// SplitMix64 for the weight initialisation.
struct Mix {
    unsigned long long s;
    unsigned long long next()
    {
        s += 0x9E3779B97F4A7C15ULL;
        unsigned long long z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

int refresh_bf16(lbpf_net* net)
{
    for (Conv& c : net->conv) {
        NK(to_bf16(net->p + c.off_w, c.wb, 9LL * c.cin * c.cout, net->stream));
        NK(flip_weights(c.wb, c.wt, c.cin, c.cout, net->stream));
    }
    return LBPF_OK;
}

}  // namespace

extern "C" int lbpf_net_create_arch(int H, int W, int batch, int levels, int base, unsigned long long seed,
                                    void* stream, lbpf_net** out)
{
    if (!out) return net_fail(nullptr, LBPF_EINVAL, "lbpf_net_create: out is NULL");
    *out = nullptr;
    if (levels < 2 || levels > 5 || !(base == 16 || base == 32 || base == 64) || (base << (levels - 1)) > 256)
        return net_fail(nullptr, LBPF_EINVAL,
                        "lbpf_net_create: levels 2..5, base 16, 32 or 64, at most 256 channels at the deepest level");
    const int q = 8 << (levels - 1);
    if (H < q || W < q || H % q || W % q || batch < 1)
        return net_fail(nullptr, LBPF_EINVAL, "lbpf_net_create: H, W must be multiples of 8 * 2^(levels - 1), batch >= 1");
    lbpf_net* net = new (std::nothrow) lbpf_net();
    if (!net) return net_fail(nullptr, LBPF_ENOMEM, "lbpf_net_create: out of host memory");
    net->H = H;
    net->W = W;
    net->N = batch;
    net->levels = levels;
    net->base = base;
    net->stream = static_cast<cudaStream_t>(stream);
    std::vector<std::pair<int, int>> cfg = {{kInPad, net->ch(0)}, {net->ch(0), net->ch(0)}};
    for (int l = 1; l < levels; ++l) {
        cfg.push_back({net->ch(l - 1), net->ch(l)});
        cfg.push_back({net->ch(l), net->ch(l)});
    }
    for (int l = levels - 2; l >= 0; --l) {
        cfg.push_back({net->ch(l + 1) + net->ch(l), net->ch(l)});
        cfg.push_back({net->ch(l), net->ch(l)});
    }
    long long off = 0, wtot = 0;
    for (auto& c2 : cfg) {
        Conv c;
        c.cin = c2.first;
        c.cout = c2.second;
        c.off_w = off;
        off += 9LL * c.cin * c.cout;
        wtot += 9LL * c.cin * c.cout;
        c.off_b = off;
        off += c.cout;
        net->conv.push_back(c);
    }
    net->off_hw = off;
    off += kOut * net->ch(0);
    net->off_hb = off;
    off += kOut;
    net->n_params = off;

    bool ok = (net->p = alloc_f(net, off)) && (net->g = alloc_f(net, off)) && (net->m = alloc_f(net, off)) &&
              (net->v = alloc_f(net, off));
    void* pb = nullptr;
    ok = ok && cudaMalloc(&pb, sizeof(__nv_bfloat16) * (size_t)wtot * 2) == cudaSuccess;
    if (pb) net->allocs.push_back(pb);
    if (ok) {
        net->pb = static_cast<__nv_bfloat16*>(pb);
        __nv_bfloat16* cur = net->pb;
        for (Conv& c : net->conv) {
            c.wb = cur;
            cur += 9LL * c.cin * c.cout;
            c.wt = cur;
            cur += 9LL * c.cin * c.cout;
        }
    }
    const long long P0 = (long long)batch * H * W;
    net->ea.assign(levels, nullptr);
    net->e.assign(levels, nullptr);
    net->pl.assign(levels, nullptr);
    net->u.assign(levels, nullptr);
    net->da.assign(levels, nullptr);
    net->d.assign(levels, nullptr);
    net->ga.assign(levels, nullptr);
    net->gb.assign(levels, nullptr);
    net->gskip.assign(levels, nullptr);
    ok = ok && (net->xin = alloc_f(net, P0 * kInPad)) && (net->out = alloc_f(net, P0 * kOut)) &&
         (net->g_out = alloc_f(net, P0 * kOut));
    for (int l = 0; l < levels && ok; ++l) {
        const long long Pl = P0 >> (2 * l);
        const int c = net->ch(l), cw = l + 1 < levels ? c + net->ch(l + 1) : c;
        ok = (net->ea[l] = alloc_f(net, Pl * c)) && (net->e[l] = alloc_f(net, Pl * c)) &&
             (net->ga[l] = alloc_f(net, Pl * cw)) && (net->gb[l] = alloc_f(net, Pl * cw));
        if (ok && l > 0) ok = (net->pl[l] = alloc_f(net, Pl * net->ch(l - 1))) != nullptr;
        if (ok && l + 1 < levels)
            ok = (net->u[l] = alloc_f(net, Pl * cw)) && (net->da[l] = alloc_f(net, Pl * c)) &&
                 (net->d[l] = alloc_f(net, Pl * c)) && (net->gskip[l] = alloc_f(net, Pl * c));
    }
    void* dl = nullptr;
    ok = ok && cudaMalloc(&dl, sizeof(double)) == cudaSuccess;
    if (dl) {
        net->allocs.push_back(dl);
        net->d_loss = static_cast<double*>(dl);
    }
    if (!ok) {
        cudaGetLastError();
        for (void* q2 : net->allocs) cudaFree(q2);
        delete net;
        return net_fail(nullptr, LBPF_ENOMEM, "lbpf_net_create: device allocation failed");
    }
    // He-uniform initialisation of the 3x3 and 1x1 weights, zero biases.
    std::vector<float> h((size_t)off, 0.f);
    Mix rng{seed};
    for (const Conv& c : net->conv) {
        const double a = std::sqrt(6.0 / (9.0 * c.cin));
        for (long long k = 0; k < 9LL * c.cin * c.cout; ++k) h[c.off_w + k] = (float)((2 * rng.uniform() - 1) * a);
    }
    for (int k = 0; k < kOut * net->ch(0); ++k) h[net->off_hw + k] = (float)((2 * rng.uniform() - 1) * 1e-2);
    if (cudaMemcpyAsync(net->p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, net->stream) !=
            cudaSuccess ||
        refresh_bf16(net) != LBPF_OK || cudaStreamSynchronize(net->stream) != cudaSuccess) {
        cudaGetLastError();
        for (void* q2 : net->allocs) cudaFree(q2);
        delete net;
        return net_fail(nullptr, LBPF_ECUDA, "lbpf_net_create: initialisation failed");
    }
    *out = net;
    return LBPF_OK;
}

extern "C" int lbpf_net_create(int H, int W, int batch, unsigned long long seed, void* stream, lbpf_net** out)
{
    return lbpf_net_create_arch(H, W, batch, 3, 16, seed, stream, out);
}

extern "C" int lbpf_net_destroy(lbpf_net* net)
{
    if (!net) return LBPF_OK;
    cudaStreamSynchronize(net->stream);
    for (void* q : net->allocs) cudaFree(q);
    delete net;
    return LBPF_OK;
}

extern "C" const char* lbpf_net_last_error(const lbpf_net* net) { return net ? net->err.c_str() : t_net_err.c_str(); }

extern "C" int lbpf_net_num_params(const lbpf_net* net, long long* n)
{
    if (!net || !n) return LBPF_EINVAL;
    *n = net->n_params;
    return LBPF_OK;
}

extern "C" int lbpf_net_get_params(lbpf_net* net, float* host, int which)
{
    if (!net || !host) return LBPF_EINVAL;
    const float* src = which == 1 ? net->g : net->p;
    NK(cudaMemcpyAsync(host, src, sizeof(float) * net->n_params, cudaMemcpyDeviceToHost, net->stream));
    NK(cudaStreamSynchronize(net->stream));
    return LBPF_OK;
}

extern "C" int lbpf_net_set_params(lbpf_net* net, const float* host)
{
    if (!net || !host) return LBPF_EINVAL;
    NK(cudaMemcpyAsync(net->p, host, sizeof(float) * net->n_params, cudaMemcpyHostToDevice, net->stream));
    int rc = refresh_bf16(net);
    if (rc) return rc;
    NK(cudaStreamSynchronize(net->stream));
    return LBPF_OK;
}

namespace {

int forward(lbpf_net* net, const float* x)
{
    const int N = net->N, H = net->H, W = net->W, lv = net->levels;
    const long long P0 = (long long)N * H * W;
    cudaStream_t s = net->stream;
    auto cv = [&](int k, const float* in, float* o, int l) -> cudaError_t {
        const Conv& c = net->conv[k];
        return conv3x3_fwd(in, c.wb, net->p + c.off_b, o, N, H >> l, W >> l, c.cin, c.cout, 1, s);
    };
    NK(pad_channels(x, net->xin, P0, kIn, kInPad, s));
    int k = 0;
    for (int l = 0; l < lv; ++l) {
        const float* a = net->xin;
        if (l > 0) {
            NK(pool_fwd(net->e[l - 1], net->pl[l], N, H >> (l - 1), W >> (l - 1), net->ch(l - 1), s));
            a = net->pl[l];
        }
        NK(cv(k, a, net->ea[l], l));
        NK(cv(k + 1, net->ea[l], net->e[l], l));
        k += 2;
    }
    const float* prev = net->e[lv - 1];
    for (int l = lv - 2; l >= 0; --l) {
        NK(upcat_fwd(prev, net->e[l], net->u[l], N, H >> l, W >> l, net->ch(l + 1), net->ch(l), s));
        NK(cv(k, net->u[l], net->da[l], l));
        NK(cv(k + 1, net->da[l], net->d[l], l));
        prev = net->d[l];
        k += 2;
    }
    NK(conv1x1_fwd(prev, net->p + net->off_hw, net->p + net->off_hb, net->out, P0, net->ch(0), kOut, s));
    NK(gate(net->xin, kInPad, net->out, P0, s));
    return LBPF_OK;
}

// Backward from g_out (dL/d out); accumulates parameter gradients into g.
// Mirrors the forward pass: decoder levels from the top down (their skip
// gradients kept), then the encoder from the deepest level up.
int backward(lbpf_net* net)
{
    const int N = net->N, H = net->H, W = net->W, lv = net->levels;
    const long long P0 = (long long)N * H * W;
    cudaStream_t s = net->stream;
    float* g = net->g;
    // through conv k at level l: dY (post-ReLU grad) given, y = its output; writes dX
    auto cvb = [&](int k, const float* in, const float* y, float* dy, float* dx, int l) -> int {
        const Conv& c = net->conv[k];
        const int h = H >> l, w = W >> l;
        const long long P = (long long)N * h * w;
        NK(relu_bwd(y, dy, P * c.cout, s));
        NK(conv3x3_wgrad(in, dy, g + c.off_w, N, h, w, c.cin, c.cout, s));
        NK(bias_grad(dy, g + c.off_b, P, c.cout, s));
        if (dx) NK(conv3x3_fwd(dy, c.wt, nullptr, dx, N, h, w, c.cout, c.cin, 0, s));
        return LBPF_OK;
    };
    int rc;
    NK(gate(net->xin, kInPad, net->g_out, P0, s));  // the gate is linear in the output
    NK(conv1x1_bwd(net->top(), net->g_out, net->p + net->off_hw, net->ga[0], g + net->off_hw, g + net->off_hb, P0,
                   net->ch(0), kOut, s));
    int k = (int)net->conv.size();
    for (int l = 0; l + 1 < lv; ++l) {  // decoder: the gradient of d[l] is in ga[l]
        k -= 2;
        if ((rc = cvb(k + 1, net->da[l], net->d[l], net->ga[l], net->gb[l], l))) return rc;
        if ((rc = cvb(k, net->u[l], net->da[l], net->gb[l], net->ga[l], l))) return rc;
        // u[l] = [up(level l + 1 output), e[l]]
        NK(upcat_bwd(net->ga[l], net->ga[l + 1], net->gskip[l], N, H >> l, W >> l, net->ch(l + 1), net->ch(l), s));
    }
    for (int l = lv - 1; l >= 0; --l) {  // encoder: the gradient of e[l] is in ga[l]
        k -= 2;
        const long long Pl = P0 >> (2 * l);
        if (l + 1 < lv) NK(add_inplace(net->ga[l], net->gskip[l], Pl * net->ch(l), s));
        if ((rc = cvb(k + 1, net->ea[l], net->e[l], net->ga[l], net->gb[l], l))) return rc;
        if ((rc = cvb(k, l > 0 ? net->pl[l] : net->xin, net->ea[l], net->gb[l], l > 0 ? net->ga[l] : nullptr, l)))
            return rc;
        if (l > 0) NK(pool_bwd(net->ga[l], net->ga[l - 1], N, H >> (l - 1), W >> (l - 1), net->ch(l - 1), s));
    }
    return LBPF_OK;
}

}  // namespace

extern "C" int lbpf_net_forward(lbpf_net* net, const float* x, float* y)
{
    if (!net || !x) return LBPF_EINVAL;
    int rc = forward(net, x);
    if (rc) return rc;
    if (y)
        NK(cudaMemcpyAsync(y, net->out, sizeof(float) * (size_t)net->N * net->H * net->W * kOut,
                           cudaMemcpyDeviceToDevice, net->stream));
    return LBPF_OK;
}

extern "C" int lbpf_net_backward(lbpf_net* net, const float* dy)
{
    if (!net || !dy) return LBPF_EINVAL;
    NK(cudaMemsetAsync(net->g, 0, sizeof(float) * net->n_params, net->stream));
    NK(cudaMemcpyAsync(net->g_out, dy, sizeof(float) * (size_t)net->N * net->H * net->W * kOut,
                       cudaMemcpyDeviceToDevice, net->stream));
    return backward(net);
}

extern "C" int lbpf_net_set_loss_weight(lbpf_net* net, float alpha)
{
    if (!net || !(alpha >= 0.f)) return LBPF_EINVAL;
    net->loss_alpha = alpha;
    return LBPF_OK;
}

extern "C" int lbpf_net_train_step(lbpf_net* net, const float* x, const float* target, float lr, double* loss)
{
    if (!net || !x || !target) return LBPF_EINVAL;
    int rc = forward(net, x);
    if (rc) return rc;
    const long long n = (long long)net->N * net->H * net->W * kOut;
    NK(cudaMemsetAsync(net->d_loss, 0, sizeof(double), net->stream));
    NK(mse(net->out, target, x, kIn, kOut, net->loss_alpha, net->g_out, net->d_loss, n, net->stream));
    NK(cudaMemsetAsync(net->g, 0, sizeof(float) * net->n_params, net->stream));
    if ((rc = backward(net))) return rc;
    net->adam_t += 1;
    NK(adam(net->p, net->g, net->m, net->v, nullptr, net->n_params, lr, 0.9f, 0.999f, 1e-8f, net->adam_t, net->stream));
    if ((rc = refresh_bf16(net))) return rc;
    if (loss) {
        NK(cudaMemcpyAsync(loss, net->d_loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
        NK(cudaStreamSynchronize(net->stream));
        if (conv_error() != 0) return net_fail(net, LBPF_ETIMEOUT, "a convolution block's bounded wait gave up");
    }
    return LBPF_OK;
}

extern "C" int lbpf_net_assemble(const float* phi, const float* u, const int* index, const float* crystal_tab,
                                 int n_crystals, float* x, long long sites, void* stream)
{
    if (!phi || !u || !x || sites < 1 || (n_crystals > 0 && !crystal_tab)) return LBPF_EINVAL;
    return assemble(phi, u, index, crystal_tab, n_crystals, x, sites, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? LBPF_OK
               : LBPF_ECUDA;
}

extern "C" int lbpf_net_apply(const float* y, float* phi, float* u, long long sites, void* stream)
{
    if (!y || !phi || !u || sites < 1) return LBPF_EINVAL;
    return apply(y, phi, u, sites, static_cast<cudaStream_t>(stream)) == cudaSuccess ? LBPF_OK : LBPF_ECUDA;
}

extern "C" int lbpf_net_delta(const float* phi0, const float* u0, const float* phi1, const float* u1, float* y,
                              long long sites, void* stream)
{
    if (!phi0 || !u0 || !phi1 || !u1 || !y || sites < 1) return LBPF_EINVAL;
    return delta(phi0, u0, phi1, u1, y, sites, static_cast<cudaStream_t>(stream)) == cudaSuccess ? LBPF_OK : LBPF_ECUDA;
}

extern "C" int lbpf_net_range_check(const float* phi, long long sites, float lo, float hi, unsigned int* count,
                                    void* stream)
{
    if (!phi || !count || sites < 1) return LBPF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(count, 0, sizeof(unsigned int), s) != cudaSuccess) return LBPF_ECUDA;
    return range_count(phi, sites, lo, hi, count, s) == cudaSuccess ? LBPF_OK : LBPF_ECUDA;
}

extern "C" int lbpf_nn_conv3x3(const float* x, const void* wt, const float* bias, float* y, int n, int H, int W,
                               int cin, int cout, int relu, void* stream)
{
    const int n_tiles = (cout + 255) / 256;
    if (!x || !wt || !y || n < 1 || H < 1 || W < 1 || cin < 16 || cout < 16 || cin % 16 || cout % (16 * n_tiles))
        return LBPF_EINVAL;
    return conv3x3_fwd(x, static_cast<const __nv_bfloat16*>(wt), bias, y, n, H, W, cin, cout, relu,
                       static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? LBPF_OK
               : LBPF_ECUDA;
}

extern "C" int lbpf_nn_conv3x3_wgrad(const float* x, const float* dy, float* dwt, int n, int H, int W, int cin,
                                     int cout, void* stream)
{
    if (!x || !dy || !dwt || n < 1 || H < 1 || W < 1 || cin < 16 || cout < 16 || cin % 16 || cout % 16 ||
        (cin > 256 && cin % 32))
        return LBPF_EINVAL;
    return conv3x3_wgrad(x, dy, dwt, n, H, W, cin, cout, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? LBPF_OK
               : LBPF_ECUDA;
}

extern "C" int lbpf_nn_conv_error(int* word)
{
    if (!word) return LBPF_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return LBPF_ECUDA;
    }
    *word = conv_error();
    return *word < 0 ? LBPF_ECUDA : LBPF_OK;
}
