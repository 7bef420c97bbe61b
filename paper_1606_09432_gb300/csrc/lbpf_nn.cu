// Kernels of the learned surrogate: a 2D U-Net on periodic fields, NHWC
// activations in FP32, 3x3 convolutions on the 5th-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory), the small
// layers on the CUDA cores in FP32.
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

// ---- 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores
//
// y[p][co] = act(sum_tap sum_ci x[p + tap][ci] w[tap][co][ci] + b[co]):
// D (M = 128 pixels of the flattened (n, h, w) order) x (N = a tile of at
// most 256 output channels, grid y) with K = 9 cin, one
// tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32, M = 128, N = the tile, K = 16)
// per 16 input channels of one tap, the accumulator in tensor memory (TMEM).  The K loop runs over stages (tap, block of KC input channels), two
// stage buffers in shared memory: while the tensor core works on stage s - 1,
// the 128 threads gather stage s — each thread one pixel row of A (the tap's
// neighbour, periodic in h and w, FP32 -> BF16) and the weight pieces of B
// (cp.async) — into the no-swizzle K-major layout: 8-row x 16-byte core
// matrices, rows of a core matrix 16 bytes apart, 8-row groups 128 bytes
// apart (SBO), 8-channel K slices one matrix apart (LBO).  One thread issues
// the MMAs of a stage and commits them to the stage buffer's mbarrier, which
// the gatherers of stage s + 2 wait on before they overwrite the buffer.
// The epilogue reads the accumulator rows with tcgen05.ld (warp w owns TMEM
// lanes 32w .. 32w + 31 = pixels), adds the bias, applies the ReLU and
// stores FP32.  Waits are bounded (2 s by %globaltimer); on expiry the block
// sets the error word and stops (conv_error()).

__device__ int g_conv_error;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO, SBO (bytes, multiples of 16),
// no swizzle, descriptor version 1 (bits 46-48 = 0b001)
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of phase `parity` of an mbarrier, at most ~2 s;
// false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity)
{
    const uint32_t a = smem_u32(mbar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(1000000u)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

constexpr int kConvM = 128;  // pixels per block (one TMEM lane each)

__global__ void __launch_bounds__(kConvM) conv3x3_tc_kernel(const float* __restrict__ x,
                                                            const __nv_bfloat16* __restrict__ w,
                                                            const float* __restrict__ bias, float* __restrict__ y,
                                                            long long P, int H, int W, int cin, int cout_all,
                                                            int cout, int KC, int relu, uint32_t tmem_cols)
{
    // output channels co0 .. co0 + cout of cout_all (grid y: channel tile)
    const int co0 = blockIdx.y * cout;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t a_bytes = (size_t)kConvM * KC * 2, b_bytes = (size_t)cout * KC * 2;
    auto sA = [&](int b) { return smem_raw + b * a_bytes; };
    auto sB = [&](int b) { return smem_raw + 2 * a_bytes + b * b_bytes; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    // this thread's pixel row
    const long long p = (long long)blockIdx.x * kConvM + tid;
    const bool valid = p < P;
    const long long HW = (long long)H * W;
    const long long img = valid ? p / HW : 0;
    const int rem = valid ? (int)(p - img * HW) : 0;
    const int py = rem / W, px = rem - py * W;
    const float* ximg = x + img * HW * cin;

    const int nkb = cin / KC, S = 9 * nkb;
    const uint32_t idesc = umma_idesc_bf16(kConvM, cout);
    bool ok = true;
    int issued = 0;  // stages committed
    for (int s = 0; s < S && ok; ++s) {
        const int buf = s & 1, tap = s / nkb, c0 = (s - tap * nkb) * KC;
        if (s >= 2 && !mbar_wait_bounded(&s_mbar[buf], ((s - 2) >> 1) & 1)) {
            atomicOr(&g_conv_error, 1);
            ok = false;
            break;
        }
        // A: row tid = x at the tap's neighbour, channels c0 .. c0 + KC
        {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            int yy = py + dy, xx = px + dx;
            yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
            xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
            const float4* src = reinterpret_cast<const float4*>(ximg + ((long long)yy * W + xx) * cin + c0);
            unsigned char* dst = sA(buf) + tid * 16;
            for (int k8 = 0; k8 < KC / 8; ++k8) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (valid) {
                    const float4 f0 = __ldg(src + 2 * k8), f1 = __ldg(src + 2 * k8 + 1);
                    v = make_uint4(pack_bf16(f0.x, f0.y), pack_bf16(f0.z, f0.w), pack_bf16(f1.x, f1.y),
                                   pack_bf16(f1.z, f1.w));
                }
                *reinterpret_cast<uint4*>(dst + (size_t)k8 * kConvM * 16) = v;
            }
        }
        // B: 16-byte pieces w[tap][co][c0 + 8 k8 ..] -> [k8][co]
        for (int e = tid; e < cout * (KC / 8); e += kConvM) {
            const int co = e % cout, k8 = e / cout;
            const __nv_bfloat16* g = w + ((size_t)tap * cout_all + co0 + co) * cin + c0 + 8 * k8;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             smem_u32(sB(buf) + (size_t)k8 * cout * 16 + co * 16)),
                         "l"(g));
        }
        asm volatile("cp.async.commit_group;");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sA(buf)), b0 = smem_u32(sB(buf));
            for (int k16 = 0; k16 < KC / 16; ++k16) {
                const uint64_t ad = umma_desc(a0 + k16 * 2 * kConvM * 16, kConvM * 16, 128);
                const uint64_t bd = umma_desc(b0 + k16 * 2 * cout * 16, cout * 16, 128);
                umma_bf16(tmem, ad, bd, idesc, (s > 0 || k16 > 0) ? 1u : 0u);
            }
            umma_commit(&s_mbar[buf]);
        }
        issued = s + 1;
    }
    // the last committed stage covers every MMA issued before it
    bool done = false;
    if (issued > 0) {
        const int last = issued - 1;
        done = mbar_wait_bounded(&s_mbar[last & 1], (last >> 1) & 1);
        if (!done) atomicOr(&g_conv_error, 2);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && done) {
        float* out = y + p * cout_all + co0;
        for (int c = 0; c < cout; c += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (valid) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    v[j] = __uint_as_float(r[j]) + (bias ? bias[co0 + c + j] : 0.f);
                    if (relu) v[j] = fmaxf(v[j], 0.f);
                }
                reinterpret_cast<float4*>(out + c)[0] = make_float4(v[0], v[1], v[2], v[3]);
                reinterpret_cast<float4*>(out + c)[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// Halo variant of the same convolution for images whose H is a multiple of
// 16 and W of 8 (with `resident`, every tap's weights are copied once beside
// the halo and all MMAs follow one barrier): a block owns a 16 x 8 tile (M = 128: tile row = 8-row group,
// pixel in the row = row of the core matrix), loads the 18 x 10 halo of all
// cin channels once (FP32 -> BF16, layout [k8][halo pixel][8]), and every tap
// is a descriptor over that halo: start at the tap's offset, SBO = one halo
// row (10 pixels x 16 bytes), LBO = one 8-channel slice (180 x 16 bytes).
// Only the weights stream through the two stage buffers (cp.async).
constexpr int kHaloY = 18, kHaloX = 10, kHaloP = kHaloY * kHaloX;

__global__ void __launch_bounds__(kConvM) conv3x3_halo_tc_kernel(const float* __restrict__ x,
                                                                 const __nv_bfloat16* __restrict__ w,
                                                                 const float* __restrict__ bias,
                                                                 float* __restrict__ y, int H, int W, int cin,
                                                                 int cout_all, int cout, int KC, int relu,
                                                                 uint32_t tmem_cols, int resident)
{
    const int co0 = blockIdx.y * cout;  // output channel tile
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles_x = W / 8, tiles = tiles_x * (H / 16);
    const int img = blockIdx.x / tiles, t = blockIdx.x - img * tiles;
    const int ty0 = (t / tiles_x) * 16, tx0 = (t % tiles_x) * 8;
    const size_t halo_bytes = (size_t)kHaloP * cin * 2, b_bytes = (size_t)cout * KC * 2;
    unsigned char* sH = smem_raw;
    auto sB = [&](int b) { return smem_raw + halo_bytes + b * b_bytes; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    const int k8n = cin / 8;
    if (resident) {  // every tap's weights, [tap][k8][co][8], copied beside the halo
        for (int e = tid; e < 9 * k8n * cout; e += kConvM) {
            const int co = e % cout, r = e / cout, k8 = r % k8n, tap = r / k8n;
            const __nv_bfloat16* g = w + ((size_t)tap * cout_all + co0 + co) * cin + 8 * k8;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sB(0) + (size_t)e * 16)), "l"(g));
        }
        asm volatile("cp.async.commit_group;");
    }
    // halo: (pixel, 8-channel slice) pieces, FP32 -> BF16
    const float* ximg = x + (size_t)img * H * W * cin;
    for (int e = tid; e < kHaloP * k8n; e += kConvM) {
        const int hp = e / k8n, k8 = e - hp * k8n;
        const int hy = hp / kHaloX, hx = hp - hy * kHaloX;
        int gy = ty0 + hy - 1, gx = tx0 + hx - 1;
        gy = gy < 0 ? gy + H : (gy >= H ? gy - H : gy);
        gx = gx < 0 ? gx + W : (gx >= W ? gx - W : gx);
        const float4* src = reinterpret_cast<const float4*>(ximg + ((size_t)gy * W + gx) * cin + 8 * k8);
        const float4 f0 = __ldg(src), f1 = __ldg(src + 1);
        *reinterpret_cast<uint4*>(sH + ((size_t)k8 * kHaloP + hp) * 16) =
            make_uint4(pack_bf16(f0.x, f0.y), pack_bf16(f0.z, f0.w), pack_bf16(f1.x, f1.y), pack_bf16(f1.z, f1.w));
    }
    if (resident) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    const int nkb = cin / KC, S = 9 * nkb;
    const uint32_t idesc = umma_idesc_bf16(kConvM, cout);
    const uint32_t h0 = smem_u32(sH);
    bool ok = true;
    int issued = 0;
    if (resident) {  // all MMAs after the one barrier, one commit
        if (tid == 0) {
            const uint32_t b0 = smem_u32(sB(0));
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                const uint32_t tap_off = (uint32_t)(((1 + dy) * kHaloX + (1 + dx)) * 16);
                for (int k16 = 0; k16 < cin / 16; ++k16) {
                    const uint64_t ad = umma_desc(h0 + (uint32_t)(2 * k16) * kHaloP * 16 + tap_off, kHaloP * 16,
                                                  kHaloX * 16);
                    const uint64_t bd = umma_desc(b0 + (uint32_t)((tap * k8n + 2 * k16) * cout * 16), cout * 16, 128);
                    umma_bf16(tmem, ad, bd, idesc, (tap > 0 || k16 > 0) ? 1u : 0u);
                }
            }
            umma_commit(&s_mbar[0]);
        }
        issued = 1;
    }
    for (int s = 0; s < S && ok && !resident; ++s) {
        const int buf = s & 1, tap = s / nkb, c0 = (s - tap * nkb) * KC;
        if (s >= 2 && !mbar_wait_bounded(&s_mbar[buf], ((s - 2) >> 1) & 1)) {
            atomicOr(&g_conv_error, 16);
            ok = false;
            break;
        }
        for (int e = tid; e < cout * (KC / 8); e += kConvM) {
            const int co = e % cout, k8 = e / cout;
            const __nv_bfloat16* g = w + ((size_t)tap * cout_all + co0 + co) * cin + c0 + 8 * k8;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             smem_u32(sB(buf) + (size_t)k8 * cout * 16 + co * 16)),
                         "l"(g));
        }
        asm volatile("cp.async.commit_group;");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const uint32_t tap_off = (uint32_t)(((1 + dy) * kHaloX + (1 + dx)) * 16);
            const uint32_t b0 = smem_u32(sB(buf));
            for (int k16 = 0; k16 < KC / 16; ++k16) {
                const int k8 = c0 / 8 + 2 * k16;
                const uint64_t ad = umma_desc(h0 + (uint32_t)k8 * kHaloP * 16 + tap_off, kHaloP * 16, kHaloX * 16);
                const uint64_t bd = umma_desc(b0 + k16 * 2 * cout * 16, cout * 16, 128);
                umma_bf16(tmem, ad, bd, idesc, (s > 0 || k16 > 0) ? 1u : 0u);
            }
            umma_commit(&s_mbar[buf]);
        }
        issued = s + 1;
    }
    bool done = false;
    if (issued > 0) {
        const int last = issued - 1;
        done = mbar_wait_bounded(&s_mbar[last & 1], (last >> 1) & 1);
        if (!done) atomicOr(&g_conv_error, 32);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && done) {
        const int m = tid, py = m >> 3, px = m & 7;
        float* out = y + (((size_t)img * H + ty0 + py) * W + tx0 + px) * cout_all + co0;
        for (int c = 0; c < cout; c += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = __uint_as_float(r[j]) + (bias ? bias[co0 + c + j] : 0.f);
                if (relu) v[j] = fmaxf(v[j], 0.f);
            }
            reinterpret_cast<float4*>(out + c)[0] = make_float4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<float4*>(out + c)[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// Input channels a stage: all of them up to 64, else the largest of 64, 48,
// 32, 16 dividing cin.
static int conv_kc(int cin)
{
    if (cin <= 64) return cin;
    for (int kc : {64, 48, 32, 16})
        if (cin % kc == 0) return kc;
    return 16;
}

cudaError_t conv3x3_fwd(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int N, int H, int W,
                        int cin, int cout_all, int relu, cudaStream_t s)
{
    // output channels in equal tiles of at most 256 (one MMA's N), multiples of 16
    const int n_tiles = (cout_all + 255) / 256;
    if (cin % 16 || cout_all % (16 * n_tiles) || cin < 16 || cout_all < 16 || H < 1 || W < 1)
        return cudaErrorInvalidValue;
    const int cout = cout_all / n_tiles;
    const int KC = conv_kc(cin);
    const size_t smem = 2 * ((size_t)kConvM * KC * 2 + (size_t)cout * KC * 2);
    static int attr_bytes = 0;
    if ((int)smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = (int)smem;
    }
    uint32_t cols = 32;
    while ((int)cols < cout) cols <<= 1;
    // halo tiles where the image divides into 16 x 8 tiles and the halo of
    // all channels fits beside the two weight buffers
    const size_t halo_smem = (size_t)kHaloP * cin * 2 + 2 * (size_t)cout * KC * 2;
    // every tap's weights beside the halo when both fit in 64 KB (3 blocks an
    // SM): measured 206 -> 192 us for 32 -> 32 channels at 1024^2, 45 -> 32 us
    // for a batch of 8 at 128^2; at 97 KB (64 -> 64) it was 4 % slower
    const size_t res_smem = (size_t)kHaloP * cin * 2 + 9 * (size_t)cin * cout * 2;
    const int resident = res_smem <= 64 * 1024 ? 1 : 0;
    const size_t hsm = resident ? res_smem : halo_smem;
    if (H % 16 == 0 && W % 8 == 0 && halo_smem <= 200 * 1024) {
        static int halo_attr = 0;
        if ((int)hsm > halo_attr) {
            cudaError_t e =
                cudaFuncSetAttribute(conv3x3_halo_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
            if (e != cudaSuccess) return e;
            halo_attr = (int)hsm;
        }
        const long long blocks = (long long)N * (H / 16) * (W / 8);
        conv3x3_halo_tc_kernel<<<dim3((unsigned)blocks, n_tiles), kConvM, hsm, s>>>(x, w, bias, y, H, W, cin,
                                                                                    cout_all, cout, KC, relu, cols,
                                                                                    resident);
        return cudaGetLastError();
    }
    const long long P = (long long)N * H * W;
    const long long blocks = (P + kConvM - 1) / kConvM;
    conv3x3_tc_kernel<<<dim3((unsigned)blocks, n_tiles), kConvM, smem, s>>>(x, w, bias, y, P, H, W, cin, cout_all,
                                                                            cout, KC, relu, cols);
    return cudaGetLastError();
}

int conv_error()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_conv_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return v;
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

// ---- weight gradient on the tensor cores
//
// dw[tap][co][ci] += sum_p dy[p][co] x[p + tap][ci]: per block one tap, one
// tile of 128 output channels (M; rows beyond cout are zero) and one tile of
// nci input channels (N), over a range of pixels (K) in stages of 64:
// A[co][p] = dy (BF16), B[ci][p] = x at the tap's neighbour (BF16), both
// gathered transposed into the no-swizzle K-major layout (8 pixels of one
// channel per 16-byte row of a core matrix).  Double-buffered stages,
// mbarrier completion and bounded waits as in conv3x3_tc_kernel; the block's
// partial sums leave tensor memory through tcgen05.ld and are added to dw
// with FP32 atomics.
constexpr int kWgK = 64;  // pixels a stage

__global__ void __launch_bounds__(kConvM) conv3x3_wgrad_tc_kernel(const float* __restrict__ x,
                                                                  const float* __restrict__ dy, float* dw, long long P,
                                                                  int H, int W, int cin, int cout, int nci,
                                                                  long long KP, uint32_t tmem_cols)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ long long s_q[2][kWgK];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tap = blockIdx.z;
    const int n_ntiles = cin / nci;
    const int co0 = (blockIdx.y / n_ntiles) * kConvM, ci0 = (blockIdx.y % n_ntiles) * nci;
    const long long p0 = (long long)blockIdx.x * KP, p1 = p0 + KP < P ? p0 + KP : P;
    const size_t a_bytes = (size_t)kConvM * kWgK * 2, b_bytes = (size_t)nci * kWgK * 2;
    auto sA = [&](int b) { return smem_raw + b * a_bytes; };
    auto sB = [&](int b) { return smem_raw + 2 * a_bytes + b * b_bytes; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    const int dyy = tap / 3 - 1, dxx = tap % 3 - 1;
    const long long HW = (long long)H * W;
    // A rows beyond cout stay zero: clear both A buffers once
    const int mv = cout - co0 < kConvM ? cout - co0 : kConvM;  // valid A rows
    for (int e = tid; e < (int)(2 * a_bytes / 16); e += kConvM)
        reinterpret_cast<uint4*>(smem_raw)[e] = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t idesc = umma_idesc_bf16(kConvM, nci);
    const int S = (int)((p1 - p0 + kWgK - 1) / kWgK);
    bool ok = true;
    int issued = 0;
    for (int s = 0; s < S && ok; ++s) {
        const int buf = s & 1;
        const long long pb = p0 + (long long)s * kWgK;
        if (s >= 2 && !mbar_wait_bounded(&s_mbar[buf], ((s - 2) >> 1) & 1)) {
            atomicOr(&g_conv_error, 4);
            ok = false;
            break;
        }
        if (tid < kWgK) {  // the stage's pixels and their neighbours at the tap
            const long long pp = pb + tid;
            long long q = -1;
            if (pp < p1) {
                const long long img = pp / HW;
                const int rem = (int)(pp - img * HW), py = rem / W, px = rem - py * W;
                int yy = py + dyy, xx = px + dxx;
                yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
                xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
                q = img * HW + (long long)yy * W + xx;
            }
            s_q[buf][tid] = q;
        }
        __syncthreads();
        // 16-byte pieces (channel row, 8 pixels) of A = dy and B = x at the
        // tap's neighbours.  Tiles of at least 128 channels: one row a thread,
        // its 64 pixels unrolled (more loads in flight); narrower tiles
        // spread the pieces over all threads, consecutive threads on
        // consecutive channels (measured 2.4x on 32 channels, 8-27 % slower
        // than one row a thread at 128-384)
        auto pieceA = [&](int m, int k8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const long long pp = pb + 8 * k8 + j;
                v[j] = pp < p1 ? __ldg(dy + pp * cout + co0 + m) : 0.f;
            }
            *reinterpret_cast<uint4*>(sA(buf) + (size_t)k8 * kConvM * 16 + m * 16) =
                make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
        };
        auto pieceB = [&](int n, int k8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const long long q = s_q[buf][8 * k8 + j];
                v[j] = q >= 0 ? __ldg(x + q * cin + ci0 + n) : 0.f;
            }
            *reinterpret_cast<uint4*>(sB(buf) + (size_t)k8 * nci * 16 + n * 16) = make_uint4(
                pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
        };
        if (mv == kConvM) {
#pragma unroll
            for (int k8 = 0; k8 < kWgK / 8; ++k8) pieceA(tid, k8);
        } else {
            for (int e = tid; e < mv * (kWgK / 8); e += kConvM) pieceA(e % mv, e / mv);
        }
        if (nci >= kConvM) {
            for (int n = tid; n < nci; n += kConvM)
#pragma unroll
                for (int k8 = 0; k8 < kWgK / 8; ++k8) pieceB(n, k8);
        } else {
            for (int e = tid; e < nci * (kWgK / 8); e += kConvM) pieceB(e % nci, e / nci);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sA(buf)), b0 = smem_u32(sB(buf));
            for (int k16 = 0; k16 < kWgK / 16; ++k16) {
                const uint64_t ad = umma_desc(a0 + k16 * 2 * kConvM * 16, kConvM * 16, 128);
                const uint64_t bd = umma_desc(b0 + k16 * 2 * nci * 16, nci * 16, 128);
                umma_bf16(tmem, ad, bd, idesc, (s > 0 || k16 > 0) ? 1u : 0u);
            }
            umma_commit(&s_mbar[buf]);
        }
        issued = s + 1;
    }
    bool done = false;
    if (issued > 0) {
        const int last = issued - 1;
        done = mbar_wait_bounded(&s_mbar[last & 1], (last >> 1) & 1);
        if (!done) atomicOr(&g_conv_error, 8);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && done) {
        for (int c = 0; c < nci; c += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int co = co0 + tid;  // this thread's TMEM lane = D row
            if (co < cout) {
                float* d = dw + ((size_t)tap * cout + co) * cin + ci0 + c;
#pragma unroll
                for (int j = 0; j < 8; ++j) atomicAdd(d + j, __uint_as_float(r[j]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

cudaError_t conv3x3_wgrad(const float* x, const float* dy, float* dw, int N, int H, int W, int cin, int cout,
                          cudaStream_t s)
{
    const int n_ntiles = (cin + 255) / 256;
    if (cin % 16 || cout % 16 || cin < 16 || cout < 16 || cin % (16 * n_ntiles)) return cudaErrorInvalidValue;
    const int nci = cin / n_ntiles, n_mtiles = (cout + kConvM - 1) / kConvM;
    const long long P = (long long)N * H * W;
    // about four blocks an SM in all: pixel chunks of a multiple of 64
    long long chunks = (4LL * 152 + 9 * n_mtiles * n_ntiles - 1) / (9 * n_mtiles * n_ntiles);
    long long KP = (P + chunks - 1) / chunks;
    KP = ((KP + kWgK - 1) / kWgK) * kWgK;
    chunks = (P + KP - 1) / KP;
    const size_t smem = 2 * ((size_t)kConvM * kWgK * 2 + (size_t)nci * kWgK * 2);
    static int attr_bytes = 0;
    if ((int)smem > attr_bytes) {
        cudaError_t e =
            cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = (int)smem;
    }
    uint32_t cols = 32;
    while ((int)cols < nci) cols <<= 1;
    dim3 grid((unsigned)chunks, (unsigned)(n_mtiles * n_ntiles), 9);
    conv3x3_wgrad_tc_kernel<<<grid, kConvM, smem, s>>>(x, dy, dw, P, H, W, cin, cout, nci, KP, cols);
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
