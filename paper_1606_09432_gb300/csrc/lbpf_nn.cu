// Kernels of the learned surrogate: a 2D U-Net on periodic fields, NHWC
// activations in FP32, 3x3 convolutions on the tensor cores with BF16
// operands and FP32 accumulation (mma.sync m16n8k16), weight gradients and
// the small layers on the CUDA cores in FP32.
//
// Layouts:
//   activations  x[n][h][w][c]            (c fastest), FP32
//   3x3 weights  w[tap][cout][cin]        BF16 (tap = 3 * (dy + 1) + (dx + 1))
//   weight grads dw[tap][cout][cin]       FP32
//   1x1 weights  w[cout][cin]             FP32
// Convolutions are periodic ("same" size, wrap-around), matching the periodic
// lattice Boltzmann domains.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbpf_nn.cuh"

namespace lbpf_nn {

constexpr int kTile = 8;           // 8 x 8 output pixels per block
constexpr int kHalo = kTile + 2;   // input tile with a 1-pixel halo
constexpr int kWarps = 4;          // 16 pixels per warp

__device__ __forceinline__ int wrap_i(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldmatrix_x2(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// y = act(conv3x3(x, w) + bias).  Block: 8 x 8 output pixels of one image,
// all COUT output channels; warp k owns pixels 16k .. 16k + 15 (two rows of
// the tile).  The input tile (10 x 10 x CIN) and all weights are staged in
// shared memory as BF16; rows of 8 channels (16 bytes) feed ldmatrix.
// Rows are padded by 8 BF16 to spread shared-memory banks.
template <int CIN, int COUT>
__global__ void __launch_bounds__(32 * kWarps) conv3x3_fwd_kernel(const float* __restrict__ x,
                                                                  const __nv_bfloat16* __restrict__ w,
                                                                  const float* __restrict__ bias, float* __restrict__ y,
                                                                  int H, int W, int relu)
{
    constexpr int XS = CIN + 8;  // padded pixel row of the input tile
    constexpr int WS = CIN + 8;  // padded cout row of a weight tap
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* s_x = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    __nv_bfloat16* s_w = s_x + kHalo * kHalo * XS;

    const int tiles_x = W / kTile;
    const int tile = blockIdx.x;
    const int img = blockIdx.y;
    const int ty0 = (tile / tiles_x) * kTile, tx0 = (tile % tiles_x) * kTile;
    const float* xi = x + (size_t)img * H * W * CIN;

    for (int e = threadIdx.x; e < kHalo * kHalo * CIN; e += blockDim.x) {
        const int c = e % CIN, p = e / CIN;
        const int hy = p / kHalo, hx = p % kHalo;
        const int gy = wrap_i(ty0 + hy - 1, H), gx = wrap_i(tx0 + hx - 1, W);
        s_x[p * XS + c] = __float2bfloat16_rn(xi[((size_t)gy * W + gx) * CIN + c]);
    }
    for (int e = threadIdx.x; e < 9 * COUT * CIN; e += blockDim.x) {
        const int ci = e % CIN, r = e / CIN;  // r = tap * COUT + co
        s_w[r * WS + ci] = w[e];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float acc[COUT / 8][4];
#pragma unroll
    for (int n = 0; n < COUT / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;

    // ldmatrix x4 for A (16 pixels x 16 channels): lanes 0-15 address the
    // rows (pixels) for channels k0..k0+7, lanes 16-31 for k0+8..k0+15.
    const int arow = lane & 15;
    const int apix = warp * 16 + arow;  // pixel within the 8 x 8 tile
    const int ay = apix / kTile, ax = apix % kTile;
    const int acol = (lane >> 4) * 8;
    // ldmatrix x2 for B (16 cin x 8 cout, stored cout-major): lanes 0-7 rows
    // (cout) for cin k0..k0+7, lanes 8-15 for k0+8..k0+15.
    const int brow = lane & 7;
    const int bcol = ((lane >> 3) & 1) * 8;

#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const uint32_t a_base = (uint32_t)__cvta_generic_to_shared(s_x + ((ay + 1 + dy) * kHalo + (ax + 1 + dx)) * XS + acol);
#pragma unroll
        for (int k0 = 0; k0 < CIN; k0 += 16) {
            uint32_t a0, a1, a2, a3;
            ldmatrix_x4(a_base + k0 * 2, a0, a1, a2, a3);
#pragma unroll
            for (int n = 0; n < COUT / 8; ++n) {
                uint32_t b0, b1;
                const uint32_t b_addr =
                    (uint32_t)__cvta_generic_to_shared(s_w + (tap * COUT + n * 8 + brow) * WS + k0 + bcol);
                ldmatrix_x2(b_addr, b0, b1);
                mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
            }
        }
    }

    // C fragment: rows lane/4 and lane/4 + 8 (pixels), cols 2 (lane%4) + {0,1}
    float* yi = y + (size_t)img * H * W * COUT;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int pix = warp * 16 + (lane >> 2) + half * 8;
        const int gy = ty0 + pix / kTile, gx = tx0 + pix % kTile;
        float* out = yi + ((size_t)gy * W + gx) * COUT;
#pragma unroll
        for (int n = 0; n < COUT / 8; ++n) {
            const int co = n * 8 + (lane & 3) * 2;
            float v0 = acc[n][half * 2 + 0], v1 = acc[n][half * 2 + 1];
            if (bias) {
                v0 += bias[co];
                v1 += bias[co + 1];
            }
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            *reinterpret_cast<float2*>(out + co) = make_float2(v0, v1);
        }
    }
}

template <int CIN, int COUT>
static cudaError_t conv_launch(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int N, int H, int W,
                               int relu, cudaStream_t s)
{
    const size_t smem = sizeof(__nv_bfloat16) * ((size_t)kHalo * kHalo * (CIN + 8) + 9 * COUT * (CIN + 8));
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_fwd_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((W / kTile) * (H / kTile), N);
    conv3x3_fwd_kernel<CIN, COUT><<<grid, 32 * kWarps, smem, s>>>(x, w, bias, y, H, W, relu);
    return cudaGetLastError();
}

cudaError_t conv3x3_fwd(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int N, int H, int W,
                        int cin, int cout, int relu, cudaStream_t s)
{
    if (H % kTile || W % kTile) return cudaErrorInvalidValue;
#define LBPF_NN_CASE(CI, CO) \
    if (cin == CI && cout == CO) return conv_launch<CI, CO>(x, w, bias, y, N, H, W, relu, s);
    LBPF_NN_CASE(16, 16)
    LBPF_NN_CASE(16, 32)
    LBPF_NN_CASE(32, 16)
    LBPF_NN_CASE(32, 32)
    LBPF_NN_CASE(32, 64)
    LBPF_NN_CASE(64, 32)
    LBPF_NN_CASE(64, 64)
    LBPF_NN_CASE(48, 16)
    LBPF_NN_CASE(16, 48)
    LBPF_NN_CASE(96, 32)
    LBPF_NN_CASE(32, 96)
#undef LBPF_NN_CASE
    return cudaErrorInvalidValue;
}

// Weights for the data gradient: dX = conv3x3(dY, wt) with
// wt[tap][ci][co] = w[8 - tap][co][ci] (taps flipped, channels swapped).
__global__ void flip_weights_kernel(const __nv_bfloat16* w, __nv_bfloat16* wt, int cin, int cout)
{
    const int total = 9 * cin * cout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int co = e % cout, r = e / cout;  // e indexes wt[tap][ci][co]
        const int ci = r % cin, tap = r / cin;
        wt[e] = w[((size_t)(8 - tap) * cout + co) * cin + ci];
    }
}

cudaError_t flip_weights(const __nv_bfloat16* w, __nv_bfloat16* wt, int cin, int cout, cudaStream_t s)
{
    flip_weights_kernel<<<64, 256, 0, s>>>(w, wt, cin, cout);
    return cudaGetLastError();
}

// dw[tap][co][ci] += sum over pixels p of dy[p][co] * x[p + tap][ci] (FP32).
// Block: one image row band of `rows` rows; thread t accumulates entries
// (tap, co, ci) = t, t + blockDim, ... over the band's pixels and adds them to
// dw atomically.
__global__ void conv3x3_wgrad_kernel(const float* __restrict__ x, const float* __restrict__ dy, float* dw, int N, int H,
                                     int W, int cin, int cout, int rows)
{
    const int bands = (H + rows - 1) / rows;
    const int img = blockIdx.x / bands, y0 = (blockIdx.x % bands) * rows;
    const int y1 = min(H, y0 + rows);
    const float* xi = x + (size_t)img * H * W * cin;
    const float* di = dy + (size_t)img * H * W * cout;
    const int entries = 9 * cout * cin;
    for (int e = threadIdx.x; e < entries; e += blockDim.x) {
        const int ci = e % cin, r = e / cin;
        const int co = r % cout, tap = r / cout;
        const int ddy = tap / 3 - 1, ddx = tap % 3 - 1;
        float acc = 0.f;
        for (int yy = y0; yy < y1; ++yy) {
            const int sy = wrap_i(yy + ddy, H);
            for (int xx = 0; xx < W; ++xx) {
                const int sx = wrap_i(xx + ddx, W);
                acc += di[((size_t)yy * W + xx) * cout + co] * xi[((size_t)sy * W + sx) * cin + ci];
            }
        }
        atomicAdd(&dw[e], acc);
    }
}

cudaError_t conv3x3_wgrad(const float* x, const float* dy, float* dw, int N, int H, int W, int cin, int cout,
                          cudaStream_t s)
{
    const int rows = 4;
    const int blocks = N * ((H + rows - 1) / rows);
    conv3x3_wgrad_kernel<<<blocks, 256, 0, s>>>(x, dy, dw, N, H, W, cin, cout, rows);
    return cudaGetLastError();
}

// Elementwise and small kernels -------------------------------------------------

__global__ void bias_grad_kernel(const float* dy, float* db, long long P, int c)
{
    // one block per channel
    const int ch = blockIdx.x;
    float acc = 0.f;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) acc += dy[p * c + ch];
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[ch] += red[0];
}

cudaError_t bias_grad(const float* dy, float* db, long long P, int c, cudaStream_t s)
{
    bias_grad_kernel<<<c, 256, 0, s>>>(dy, db, P, c);
    return cudaGetLastError();
}

__global__ void relu_bwd_kernel(const float* y, float* dy, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) dy[i] = 0.f;
}

static int eblocks(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

cudaError_t relu_bwd(const float* y, float* dy, long long n, cudaStream_t s)
{
    relu_bwd_kernel<<<eblocks(n), 256, 0, s>>>(y, dy, n);
    return cudaGetLastError();
}

// 2 x 2 average pool (NHWC) and its gradient.
__global__ void pool_fwd_kernel(const float* x, float* y, int N, int H, int W, int c)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Ho * Wo * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = i % c;
        long long r = i / c;
        const int xo = r % Wo;
        r /= Wo;
        const int yo = r % Ho;
        const int n = (int)(r / Ho);
        const float* b = x + (((size_t)n * H + 2 * yo) * W + 2 * xo) * c + ch;
        y[i] = 0.25f * (b[0] + b[c] + b[(size_t)W * c] + b[(size_t)W * c + c]);
    }
}

__global__ void pool_bwd_kernel(const float* dy, float* dx, int N, int H, int W, int c)
{
    const long long total = (long long)N * H * W * c;
    const int Wo = W / 2, Ho = H / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = i % c;
        long long r = i / c;
        const int xx = r % W;
        r /= W;
        const int yy = r % H;
        const int n = (int)(r / H);
        dx[i] = 0.25f * dy[(((size_t)n * Ho + yy / 2) * Wo + xx / 2) * c + ch];
    }
}

cudaError_t pool_fwd(const float* x, float* y, int N, int H, int W, int c, cudaStream_t s)
{
    pool_fwd_kernel<<<eblocks((long long)N * H * W * c / 4), 256, 0, s>>>(x, y, N, H, W, c);
    return cudaGetLastError();
}
cudaError_t pool_bwd(const float* dy, float* dx, int N, int H, int W, int c, cudaStream_t s)
{
    pool_bwd_kernel<<<eblocks((long long)N * H * W * c), 256, 0, s>>>(dy, dx, N, H, W, c);
    return cudaGetLastError();
}

// Nearest 2x upsample of `a` (N, H/2, W/2, ca) concatenated with the skip `b`
// (N, H, W, cb) into y (N, H, W, ca + cb), and the backward split.
__global__ void upcat_fwd_kernel(const float* a, const float* b, float* y, int N, int H, int W, int ca, int cb)
{
    const int c = ca + cb;
    const long long total = (long long)N * H * W * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = i % c;
        const long long p = i / c;
        const int xx = p % W;
        const long long r = p / W;
        const int yy = r % H;
        const int n = (int)(r / H);
        y[i] = ch < ca ? a[(((size_t)n * (H / 2) + yy / 2) * (W / 2) + xx / 2) * ca + ch] : b[p * cb + (ch - ca)];
    }
}

__global__ void upcat_bwd_kernel(const float* dy, float* da, float* db, int N, int H, int W, int ca, int cb)
{
    // da: sum over the 2 x 2 children; db: copy
    const int c = ca + cb;
    const long long total_a = (long long)N * (H / 2) * (W / 2) * ca;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total_a;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = i % ca;
        long long r = i / ca;
        const int xo = r % (W / 2);
        r /= (W / 2);
        const int yo = r % (H / 2);
        const int n = (int)(r / (H / 2));
        const float* b0 = dy + (((size_t)n * H + 2 * yo) * W + 2 * xo) * c + ch;
        da[i] = b0[0] + b0[c] + b0[(size_t)W * c] + b0[(size_t)W * c + c];
    }
    const long long total_b = (long long)N * H * W * cb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total_b;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = i % cb;
        const long long p = i / cb;
        db[i] = dy[p * c + ca + ch];
    }
}

cudaError_t upcat_fwd(const float* a, const float* b, float* y, int N, int H, int W, int ca, int cb, cudaStream_t s)
{
    upcat_fwd_kernel<<<eblocks((long long)N * H * W * (ca + cb)), 256, 0, s>>>(a, b, y, N, H, W, ca, cb);
    return cudaGetLastError();
}
cudaError_t upcat_bwd(const float* dy, float* da, float* db, int N, int H, int W, int ca, int cb, cudaStream_t s)
{
    upcat_bwd_kernel<<<eblocks((long long)N * H * W * cb), 256, 0, s>>>(dy, da, db, N, H, W, ca, cb);
    return cudaGetLastError();
}

// 1 x 1 convolution (FP32): y[p][co] = b[co] + sum_ci w[co][ci] x[p][ci].
__global__ void conv1x1_fwd_kernel(const float* x, const float* w, const float* b, float* y, long long P, int cin,
                                   int cout)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * cout;
         i += (long long)gridDim.x * blockDim.x) {
        const int co = i % cout;
        const long long p = i / cout;
        float acc = b[co];
        for (int ci = 0; ci < cin; ++ci) acc += w[co * cin + ci] * x[p * cin + ci];
        y[i] = acc;
    }
}

// dx[p][ci] = sum_co w[co][ci] dy[p][co]
__global__ void conv1x1_dgrad_kernel(const float* dy, const float* w, float* dx, long long P, int cin, int cout)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * cin;
         i += (long long)gridDim.x * blockDim.x) {
        const int ci = i % cin;
        const long long p = i / cin;
        float acc = 0.f;
        for (int co = 0; co < cout; ++co) acc += w[co * cin + ci] * dy[p * cout + co];
        dx[i] = acc;
    }
}

// dw[co][ci] += sum_p dy[p][co] x[p][ci]; one block per (co, ci).
__global__ void conv1x1_wgrad_kernel(const float* x, const float* dy, float* dw, long long P, int cin, int cout)
{
    const int co = blockIdx.x / cin, ci = blockIdx.x % cin;
    float acc = 0.f;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) acc += dy[p * cout + co] * x[p * cin + ci];
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) dw[blockIdx.x] += red[0];
}

cudaError_t conv1x1_fwd(const float* x, const float* w, const float* b, float* y, long long P, int cin, int cout,
                        cudaStream_t s)
{
    conv1x1_fwd_kernel<<<eblocks(P * cout), 256, 0, s>>>(x, w, b, y, P, cin, cout);
    return cudaGetLastError();
}
cudaError_t conv1x1_bwd(const float* x, const float* dy, const float* w, float* dx, float* dw, float* db, long long P,
                        int cin, int cout, cudaStream_t s)
{
    if (dx) conv1x1_dgrad_kernel<<<eblocks(P * cin), 256, 0, s>>>(dy, w, dx, P, cin, cout);
    conv1x1_wgrad_kernel<<<cin * cout, 256, 0, s>>>(x, dy, dw, P, cin, cout);
    bias_grad_kernel<<<cout, 256, 0, s>>>(dy, db, P, cout);
    return cudaGetLastError();
}

// Weighted mean squared error over n values (cout per site): loss[0] +=
// sum w (p - t)^2 / n (FP64 atomics per block), dp = 2 w (p - t) / n, with
// w = 1 + alpha max(0, 1 - phi^2) and phi = x[site * cin] the input phase
// field of the value's site (alpha = 0: plain mean squared error).
__global__ void mse_kernel(const float* p, const float* t, const float* x, int cin, int cout, float alpha, float* dp,
                           double* loss, long long n)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = p[i] - t[i];
        float w = 1.f;
        if (alpha > 0.f) {
            const float ph = x[(i / cout) * cin];
            w += alpha * fmaxf(0.f, 1.f - ph * ph);
        }
        dp[i] = 2.f * w * d / (float)n;
        acc += (double)w * d * d;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)n);
}

cudaError_t mse(const float* p, const float* t, const float* x, int cin, int cout, float alpha, float* dp, double* loss,
                long long n, cudaStream_t s)
{
    mse_kernel<<<eblocks(n) < 304 ? eblocks(n) : 304, 256, 0, s>>>(p, t, x, cin, cout, alpha, dp, loss, n);
    return cudaGetLastError();
}

// Adam update of FP32 master weights; refreshes the BF16 copy when given.
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, __nv_bfloat16* wb, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

cudaError_t adam(float* w, const float* g, float* m, float* v, __nv_bfloat16* wb, long long n, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t s)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<eblocks(n), 256, 0, s>>>(w, g, m, v, wb, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

__global__ void to_bf16_kernel(const float* a, __nv_bfloat16* b, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

cudaError_t to_bf16(const float* a, __nv_bfloat16* b, long long n, cudaStream_t s)
{
    to_bf16_kernel<<<eblocks(n), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

// Pad NHWC channels: y[p][c] = c < cin ? x[p][c] : 0 (cout >= cin).
__global__ void pad_channels_kernel(const float* x, float* y, long long P, int cin, int cout)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * cout;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = i % cout;
        y[i] = c < cin ? x[(i / cout) * cin + c] : 0.f;
    }
}

cudaError_t pad_channels(const float* x, float* y, long long P, int cin, int cout, cudaStream_t s)
{
    pad_channels_kernel<<<eblocks(P * cout), 256, 0, s>>>(x, y, P, cin, cout);
    return cudaGetLastError();
}

}  // namespace lbpf_nn

namespace lbpf_nn {

__global__ void add_kernel(float* a, const float* b, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] += b[i];
}

cudaError_t add_inplace(float* a, const float* b, long long n, cudaStream_t s)
{
    add_kernel<<<eblocks(n), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

}  // namespace lbpf_nn

namespace lbpf_nn {

// x[p] = (phi, u, cos 4 theta, sin 4 theta, eps) of the site's crystal
// (crystal table tab[2 * (I - 1)] = eps, tab[2 * (I - 1) + 1] = theta; I from
// the index field, 1 everywhere when index is NULL; zeros where I = 0).
__global__ void assemble_kernel(const float* phi, const float* u, const int* index, const float* tab, int nc, float* x,
                                long long P)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int I = index ? index[p] : 1;
        float c = 0.f, sn = 0.f, e = 0.f;
        if (I >= 1 && I <= nc) {
            e = tab[2 * (I - 1)];
            sincosf(4.f * tab[2 * (I - 1) + 1], &sn, &c);
        }
        float* o = x + p * 5;
        o[0] = phi[p];
        o[1] = u[p];
        o[2] = c;
        o[3] = sn;
        o[4] = e;
    }
}

cudaError_t assemble(const float* phi, const float* u, const int* index, const float* tab, int nc, float* x, long long P,
                     cudaStream_t s)
{
    assemble_kernel<<<eblocks(P), 256, 0, s>>>(phi, u, index, tab, nc, x, P);
    return cudaGetLastError();
}

// phi += y[p][0], u += y[p][1]
__global__ void apply_kernel(const float* y, float* phi, float* u, long long P)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        phi[p] += y[2 * p];
        u[p] += y[2 * p + 1];
    }
}

cudaError_t apply(const float* y, float* phi, float* u, long long P, cudaStream_t s)
{
    apply_kernel<<<eblocks(P), 256, 0, s>>>(y, phi, u, P);
    return cudaGetLastError();
}

}  // namespace lbpf_nn

namespace lbpf_nn {

// y[p] = (phi1 - phi0, u1 - u0): training target of a jump.
__global__ void delta_kernel(const float* phi0, const float* u0, const float* phi1, const float* u1, float* y,
                             long long P)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        y[2 * p] = phi1[p] - phi0[p];
        y[2 * p + 1] = u1[p] - u0[p];
    }
}

cudaError_t delta(const float* phi0, const float* u0, const float* phi1, const float* u1, float* y, long long P,
                  cudaStream_t s)
{
    delta_kernel<<<eblocks(P), 256, 0, s>>>(phi0, u0, phi1, u1, y, P);
    return cudaGetLastError();
}

// count[0] += number of phi values outside [lo, hi] (or not finite).
__global__ void range_kernel(const float* phi, long long P, float lo, float hi, unsigned int* count)
{
    unsigned int c = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x)
        if (!(phi[p] >= lo && phi[p] <= hi)) ++c;
    if (c) atomicAdd(count, c);
}

cudaError_t range_count(const float* phi, long long P, float lo, float hi, unsigned int* count, cudaStream_t s)
{
    range_kernel<<<eblocks(P) < 608 ? eblocks(P) : 608, 256, 0, s>>>(phi, P, lo, hi, count);
    return cudaGetLastError();
}

}  // namespace lbpf_nn

namespace lbpf_nn {

// Interface gate of the phi output: out[p][0] *= 1 - x[p][0]^2 (x channel 0 is
// phi), so that the network changes phi only in the diffuse interface.  The
// same factor scales the gradient.
__global__ void gate_kernel(const float* x, int cx, float* out, long long P)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float ph = x[p * cx];
        out[2 * p] *= (1.f - ph) * (1.f + ph);
    }
}

cudaError_t gate(const float* x, int cx, float* out, long long P, cudaStream_t s)
{
    gate_kernel<<<eblocks(P), 256, 0, s>>>(x, cx, out, P);
    return cudaGetLastError();
}

}  // namespace lbpf_nn
