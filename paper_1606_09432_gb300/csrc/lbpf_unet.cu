// The learned surrogate's network runtime: a 2D U-Net with three levels
// (16, 32, 64 channels), periodic 3x3 convolutions + ReLU, 2x2 average
// pooling, nearest 2x upsampling with skip concatenation and a 1x1 head.
// Input per site: (phi, u, cos 4 theta, sin 4 theta, eps) zero-padded to 16
// channels; output: (d phi, d u), the change of phi and u over the jump, the
// phi channel gated by (1 - phi^2) so that the bulk phases stay untouched.
// Forward, hand-written backward and Adam run in the kernels of lbpf_nn.cu.
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
    int H = 0, W = 0, N = 0;
    cudaStream_t stream = nullptr;
    std::vector<Conv> conv;  // 10 3x3 convolutions in forward order
    long long off_hw = 0, off_hb = 0, n_params = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 params, grads, Adam moments
    __nv_bfloat16* pb = nullptr;  // BF16 copy of all params (only 3x3 parts used)
    int adam_t = 0;
    float loss_alpha = 0.f;  // interface weight of the training loss
    // activations (N, h, w, c) and their gradients
    float *xin, *a1a, *a1, *p1, *a2a, *a2, *p2, *a3a, *a3, *u2, *d2a, *d2, *u1, *d1a, *d1, *out;
    float *g_big0, *g_big1, *g_mid0, *g_mid1, *g_sml0, *g_sml1, *g_cat1, *g_cat2, *g_out;
    double* d_loss = nullptr;
    std::vector<void*> allocs;
    std::string err;
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
    if (cudaMalloc(&p, sizeof(float) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    net->allocs.push_back(p);
    cudaMemsetAsync(p, 0, sizeof(float) * (size_t)n, net->stream);
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

extern "C" int lbpf_net_create(int H, int W, int batch, unsigned long long seed, void* stream, lbpf_net** out)
{
    if (!out) return net_fail(nullptr, LBPF_EINVAL, "lbpf_net_create: out is NULL");
    *out = nullptr;
    if (H < 32 || W < 32 || H % 32 || W % 32 || batch < 1)
        return net_fail(nullptr, LBPF_EINVAL, "lbpf_net_create: H, W must be multiples of 32 (>= 32), batch >= 1");
    lbpf_net* net = new (std::nothrow) lbpf_net();
    if (!net) return net_fail(nullptr, LBPF_ENOMEM, "lbpf_net_create: out of host memory");
    net->H = H;
    net->W = W;
    net->N = batch;
    net->stream = static_cast<cudaStream_t>(stream);
    const int cfg[10][2] = {{16, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64}, {96, 32}, {32, 32}, {48, 16}, {16, 16}};
    long long off = 0;
    for (auto& c2 : cfg) {
        Conv c;
        c.cin = c2[0];
        c.cout = c2[1];
        c.off_w = off;
        off += 9LL * c.cin * c.cout;
        c.off_b = off;
        off += c.cout;
        net->conv.push_back(c);
    }
    net->off_hw = off;
    off += kOut * 16;
    net->off_hb = off;
    off += kOut;
    net->n_params = off;

    const long long P1 = (long long)batch * H * W, P2 = P1 / 4, P3 = P1 / 16;
    bool ok = (net->p = alloc_f(net, off)) && (net->g = alloc_f(net, off)) && (net->m = alloc_f(net, off)) &&
              (net->v = alloc_f(net, off));
    void* pb = nullptr;
    ok = ok && cudaMalloc(&pb, sizeof(__nv_bfloat16) * (size_t)off * 2) == cudaSuccess;
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
    ok = ok && (net->xin = alloc_f(net, P1 * kInPad)) && (net->a1a = alloc_f(net, P1 * 16)) &&
         (net->a1 = alloc_f(net, P1 * 16)) && (net->p1 = alloc_f(net, P2 * 16)) && (net->a2a = alloc_f(net, P2 * 32)) &&
         (net->a2 = alloc_f(net, P2 * 32)) && (net->p2 = alloc_f(net, P3 * 32)) && (net->a3a = alloc_f(net, P3 * 64)) &&
         (net->a3 = alloc_f(net, P3 * 64)) && (net->u2 = alloc_f(net, P2 * 96)) && (net->d2a = alloc_f(net, P2 * 32)) &&
         (net->d2 = alloc_f(net, P2 * 32)) && (net->u1 = alloc_f(net, P1 * 48)) && (net->d1a = alloc_f(net, P1 * 16)) &&
         (net->d1 = alloc_f(net, P1 * 16)) && (net->out = alloc_f(net, P1 * kOut));
    ok = ok && (net->g_big0 = alloc_f(net, P1 * 16)) && (net->g_big1 = alloc_f(net, P1 * 16)) &&
         (net->g_mid0 = alloc_f(net, P2 * 32)) && (net->g_mid1 = alloc_f(net, P2 * 32)) &&
         (net->g_sml0 = alloc_f(net, P3 * 64)) && (net->g_sml1 = alloc_f(net, P3 * 64)) &&
         (net->g_cat1 = alloc_f(net, P1 * 48)) && (net->g_cat2 = alloc_f(net, P2 * 96)) &&
         (net->g_out = alloc_f(net, P1 * kOut));
    void* dl = nullptr;
    ok = ok && cudaMalloc(&dl, sizeof(double)) == cudaSuccess;
    if (dl) {
        net->allocs.push_back(dl);
        net->d_loss = static_cast<double*>(dl);
    }
    if (!ok) {
        cudaGetLastError();
        for (void* q : net->allocs) cudaFree(q);
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
    for (int k = 0; k < kOut * 16; ++k) h[net->off_hw + k] = (float)((2 * rng.uniform() - 1) * 1e-2);
    if (cudaMemcpyAsync(net->p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, net->stream) !=
            cudaSuccess ||
        refresh_bf16(net) != LBPF_OK || cudaStreamSynchronize(net->stream) != cudaSuccess) {
        cudaGetLastError();
        for (void* q : net->allocs) cudaFree(q);
        delete net;
        return net_fail(nullptr, LBPF_ECUDA, "lbpf_net_create: initialisation failed");
    }
    *out = net;
    return LBPF_OK;
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
    const int N = net->N, H = net->H, W = net->W;
    const long long P1 = (long long)N * H * W;
    cudaStream_t s = net->stream;
    auto cv = [&](int k, const float* in, float* o, int h, int w) -> cudaError_t {
        const Conv& c = net->conv[k];
        return conv3x3_fwd(in, c.wb, net->p + c.off_b, o, N, h, w, c.cin, c.cout, 1, s);
    };
    NK(pad_channels(x, net->xin, P1, kIn, kInPad, s));
    NK(cv(0, net->xin, net->a1a, H, W));
    NK(cv(1, net->a1a, net->a1, H, W));
    NK(pool_fwd(net->a1, net->p1, N, H, W, 16, s));
    NK(cv(2, net->p1, net->a2a, H / 2, W / 2));
    NK(cv(3, net->a2a, net->a2, H / 2, W / 2));
    NK(pool_fwd(net->a2, net->p2, N, H / 2, W / 2, 32, s));
    NK(cv(4, net->p2, net->a3a, H / 4, W / 4));
    NK(cv(5, net->a3a, net->a3, H / 4, W / 4));
    NK(upcat_fwd(net->a3, net->a2, net->u2, N, H / 2, W / 2, 64, 32, s));
    NK(cv(6, net->u2, net->d2a, H / 2, W / 2));
    NK(cv(7, net->d2a, net->d2, H / 2, W / 2));
    NK(upcat_fwd(net->d2, net->a1, net->u1, N, H, W, 32, 16, s));
    NK(cv(8, net->u1, net->d1a, H, W));
    NK(cv(9, net->d1a, net->d1, H, W));
    NK(conv1x1_fwd(net->d1, net->p + net->off_hw, net->p + net->off_hb, net->out, P1, 16, kOut, s));
    NK(gate(net->xin, kInPad, net->out, P1, s));
    return LBPF_OK;
}

// Backward from g_out (dL/d out); accumulates parameter gradients into g.
int backward(lbpf_net* net)
{
    const int N = net->N, H = net->H, W = net->W;
    const long long P1 = (long long)N * H * W, P2 = P1 / 4, P3 = P1 / 16;
    cudaStream_t s = net->stream;
    float* g = net->g;
    // through conv k: dY (post-ReLU grad) given, y = its output; writes dX
    auto cvb = [&](int k, const float* in, const float* y, float* dy, float* dx, int h, int w, long long P) -> int {
        const Conv& c = net->conv[k];
        NK(relu_bwd(y, dy, P * c.cout, s));
        NK(conv3x3_wgrad(in, dy, g + c.off_w, N, h, w, c.cin, c.cout, s));
        NK(bias_grad(dy, g + c.off_b, P, c.cout, s));
        if (dx) NK(conv3x3_fwd(dy, c.wt, nullptr, dx, N, h, w, c.cout, c.cin, 0, s));
        return LBPF_OK;
    };
    int rc;
    NK(gate(net->xin, kInPad, net->g_out, P1, s));  // the gate is linear in the output
    NK(conv1x1_bwd(net->d1, net->g_out, net->p + net->off_hw, net->g_big0, g + net->off_hw, g + net->off_hb, P1, 16,
                   kOut, s));
    if ((rc = cvb(9, net->d1a, net->d1, net->g_big0, net->g_big1, H, W, P1))) return rc;
    if ((rc = cvb(8, net->u1, net->d1a, net->g_big1, net->g_cat1, H, W, P1))) return rc;
    // u1 = [up(d2) (32), a1 (16)]
    NK(upcat_bwd(net->g_cat1, net->g_mid0, net->g_big0, N, H, W, 32, 16, s));  // g_big0 = da1 (skip part)
    if ((rc = cvb(7, net->d2a, net->d2, net->g_mid0, net->g_mid1, H / 2, W / 2, P2))) return rc;
    if ((rc = cvb(6, net->u2, net->d2a, net->g_mid1, net->g_cat2, H / 2, W / 2, P2))) return rc;
    // u2 = [up(a3) (64), a2 (32)]
    NK(upcat_bwd(net->g_cat2, net->g_sml0, net->g_mid0, N, H / 2, W / 2, 64, 32, s));  // g_mid0 = da2 (skip part)
    if ((rc = cvb(5, net->a3a, net->a3, net->g_sml0, net->g_sml1, H / 4, W / 4, P3))) return rc;
    if ((rc = cvb(4, net->p2, net->a3a, net->g_sml1, net->g_sml0, H / 4, W / 4, P3))) return rc;  // g_sml0 = dp2
    NK(pool_bwd(net->g_sml0, net->g_mid1, N, H / 2, W / 2, 32, s));
    NK(add_inplace(net->g_mid0, net->g_mid1, P2 * 32, s));  // da2 total
    if ((rc = cvb(3, net->a2a, net->a2, net->g_mid0, net->g_mid1, H / 2, W / 2, P2))) return rc;
    if ((rc = cvb(2, net->p1, net->a2a, net->g_mid1, net->g_mid0, H / 2, W / 2, P2))) return rc;  // g_mid0 = dp1 (16 ch)
    NK(pool_bwd(net->g_mid0, net->g_big1, N, H, W, 16, s));
    NK(add_inplace(net->g_big0, net->g_big1, P1 * 16, s));  // da1 total
    if ((rc = cvb(1, net->a1a, net->a1, net->g_big0, net->g_big1, H, W, P1))) return rc;
    if ((rc = cvb(0, net->xin, net->a1a, net->g_big1, nullptr, H, W, P1))) return rc;
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
    if (!x || !wt || !y || n < 1 || H < 1 || W < 1 || cin < 16 || cout < 16 || cin % 16 || cout % 16 || cout > 256)
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
