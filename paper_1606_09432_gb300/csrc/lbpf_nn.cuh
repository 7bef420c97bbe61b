// Declarations of the surrogate network's kernels (lbpf_nn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lbpf_nn {

// y = act(conv3x3(x, w) + bias), periodic padding, on the tensor cores
// (tcgen05); cin a multiple of 16; cout in equal tiles of at most 256
// channels, each a multiple of 16.  w: BF16 [tap][cout][cin].
cudaError_t conv3x3_fwd(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int N, int H, int W,
                        int cin, int cout, int relu, cudaStream_t s);
// Error word of the convolution kernels (1, 2: a bounded wait of a block
// gave up; -1: unreadable); 0 when every wait completed.
int conv_error();
// wt[tap][ci][co] = w[8 - tap][co][ci]: weights of the data-gradient convolution.
cudaError_t flip_weights(const __nv_bfloat16* w, __nv_bfloat16* wt, int cin, int cout, cudaStream_t s);
// dw[tap][co][ci] += sum_p dy[p][co] x[p + tap][ci], BF16 operands on the tensor
// cores, FP32 accumulation; cin, cout multiples of 16 (cin > 256: of 32).
cudaError_t conv3x3_wgrad(const float* x, const float* dy, float* dw, int N, int H, int W, int cin, int cout,
                          cudaStream_t s);
cudaError_t bias_grad(const float* dy, float* db, long long P, int c, cudaStream_t s);
cudaError_t relu_bwd(const float* y, float* dy, long long n, cudaStream_t s);
cudaError_t pool_fwd(const float* x, float* y, int N, int H, int W, int c, cudaStream_t s);
cudaError_t pool_bwd(const float* dy, float* dx, int N, int H, int W, int c, cudaStream_t s);
cudaError_t upcat_fwd(const float* a, const float* b, float* y, int N, int H, int W, int ca, int cb, cudaStream_t s);
cudaError_t upcat_bwd(const float* dy, float* da, float* db, int N, int H, int W, int ca, int cb, cudaStream_t s);
cudaError_t conv1x1_fwd(const float* x, const float* w, const float* b, float* y, long long P, int cin, int cout,
                        cudaStream_t s);
cudaError_t conv1x1_bwd(const float* x, const float* dy, const float* w, float* dx, float* dw, float* db, long long P,
                        int cin, int cout, cudaStream_t s);
cudaError_t mse(const float* p, const float* t, const float* x, int cin, int cout, float alpha, float* dp, double* loss,
                long long n, cudaStream_t s);
cudaError_t adam(float* w, const float* g, float* m, float* v, __nv_bfloat16* wb, long long n, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t s);
cudaError_t to_bf16(const float* a, __nv_bfloat16* b, long long n, cudaStream_t s);
cudaError_t pad_channels(const float* x, float* y, long long P, int cin, int cout, cudaStream_t s);
cudaError_t add_inplace(float* a, const float* b, long long n, cudaStream_t s);
cudaError_t assemble(const float* phi, const float* u, const int* index, const float* tab, int nc, float* x, long long P,
                     cudaStream_t s);
cudaError_t apply(const float* y, float* phi, float* u, long long P, cudaStream_t s);
cudaError_t delta(const float* phi0, const float* u0, const float* phi1, const float* u1, float* y, long long P,
                  cudaStream_t s);
cudaError_t gate(const float* x, int cx, float* out, long long P, cudaStream_t s);
cudaError_t range_count(const float* phi, long long P, float lo, float hi, unsigned int* count, cudaStream_t s);

}  // namespace lbpf_nn
