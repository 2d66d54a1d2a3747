// Tensor-core convolutions of the learned stage (sm_103a, tcgen05).
//
// A 3x3 convolution is the contraction D[m][n] = sum_k A[m][k] B[n][k] with
// m an output pixel, n an output channel and k = (input channel, ky, kx):
// A is the input gathered around each pixel (implicit im2col), B the weights.
// The input gradient of a convolution is the same contraction with m an input
// pixel, n an input channel, k = (output channel, ky, kx), A the output
// gradient gathered through the transposed stencil and B the weights read
// transposed.
// One CTA of 128 threads computes 128 consecutive output pixels (M = 128) for
// all output channels (N = Cout rounded up to 16, 32 or 64).  K advances 16 at
// a time: every thread gathers its pixel's 16 values of A (bfloat16) into a
// shared-memory stage, the threads fill B, and one elected thread issues
// tcgen05.mma (kind::f16, bfloat16 operands, float32 accumulator in tensor
// memory) and commits it to the stage's mbarrier.  Two stages alternate, so
// the gather of step k + 1 overlaps the MMA of step k.  The epilogue reads the
// accumulator rows back with tcgen05.ld (warp w owns tensor-memory lanes
// 32w .. 32w + 31, i.e. pixels 32w .. 32w + 31 of the tile), adds the bias and
// applies relu / the skip connection.
//
// Shared-memory operands use the no-swizzle K-major layout: 8 x 16-byte core
// matrices (8 rows, 8 bfloat16 along K), consecutive along K at LBO = 128 B
// and along M (or N) at SBO = 256 B, so one K = 16 step of A is 4 KB and of B
// NT x 32 B.
//
// Every wait on an mbarrier is bounded; on timeout the kernel sets *err, waits
// (bounded) for its last commit, frees its tensor memory and leaves without
// writing its outputs.
#include <cstdint>

#include "mxp_internal.h"

namespace mxp {

constexpr long long kMbarPollLimit = 1ll << 22;   // try_wait polls (each suspends briefly): well over a second

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kMbarPollLimit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // start address, leading (K) and stride (M / N) byte offsets in 16-byte
    // units, descriptor version 1, no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: float32 accumulator, bfloat16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

constexpr uint32_t kLBO = 128, kSBO = 256;

// byte offset of element (row, k) (k < 16) of a no-swizzle K-major operand stage
__device__ __forceinline__ uint32_t kmajor_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// MODE 0, forward convolution (see cnn.cu for the network):
//   out[n, co, oy, ox] = act(bias[co] + sum_{ci, ky, kx} W[co, ci, ky, kx] x[n, ci, S oy + ky - 1, S ox + kx - 1])
//   with x the logical input (nearest-upsampled by 2 when UPS) and zero padding;
//   out_skip (nullable) = out + skip.  in = x [n][Cin][Hs][Ws], out [n][Cout][Ho][Wo].
// MODE 1, input gradient of that convolution (UPS = 0):
//   out[n, ci, y, x] = sum_{co, ky, kx} W[co, ci, ky, kx] g[n, co, (y + 1 - ky) / S, (x + 1 - kx) / S]
//   over the terms whose division is exact and in range.  in = g [n][Cin][Hs][Ws]
//   (Cin = the layer's output channels), out [n][Cout][Ho][Wo] (Cout = the
//   layer's input channels, Ho x Wo its logical input size); no bias or relu.
template <int MODE, int S, int UPS, int NT>
__global__ void __launch_bounds__(128) k_conv_tc(const float *__restrict__ in, int Cin, int Hs, int Ws,
                                                 const __nv_bfloat16 *__restrict__ w,
                                                 const float *__restrict__ bias, int Cout, int Ho, int Wo,
                                                 int relu, const float *__restrict__ skip,
                                                 float *__restrict__ out, float *__restrict__ out_skip,
                                                 int64_t npix, unsigned *err)
{
    static_assert(MODE == 0 || (MODE == 1 && UPS == 0), "the input gradient takes no upsampling");
    static_assert(NT == 16 || NT == 32 || NT == 64, "N tile of 16, 32 or 64 channels");
    constexpr int TCOLS = NT < 32 ? 32 : NT;        // tensor-memory columns (power of two, >= 32)
    __shared__ __align__(128) uint8_t sA[2][4096];
    __shared__ __align__(128) uint8_t sB[2][NT * 32];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    // this thread's output pixel (row of A and of D)
    const int64_t m = (int64_t)blockIdx.x * 128 + tid;
    const bool mvalid = m < npix;
    const int64_t hw = (int64_t)Ho * Wo;
    const int img = mvalid ? (int)(m / hw) : 0;
    const int rr = mvalid ? (int)(m % hw) : 0;
    const int oy = rr / Wo, ox = rr % Wo;
    const int Hl = UPS ? 2 * Hs : Hs, Wl = UPS ? 2 * Ws : Ws;
    const float *xin = in + (int64_t)img * Cin * Hs * Ws;
    const int K = Cin * 9;
    const int nk = (K + 15) / 16;
    constexpr uint32_t idesc = umma_idesc_bf16(128, NT);
    bool ok = true;
    int issued = 0;                          // K steps whose MMA was issued (uniform over the CTA)
    for (int kc = 0; kc < nk; ++kc) {
        const int stage = kc & 1;
        bool free_ok = true;
        if (kc >= 2) free_ok = mbar_wait(&mbar[stage], ((kc - 2) >> 1) & 1);   // MMA of step kc - 2 done
        ok = __syncthreads_and(free_ok) != 0;
        if (!ok) break;
        // A: 16 gathered input values of this pixel
        uint32_t packed[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = kc * 16 + 2 * q + h;
                float v = 0.f;
                if (mvalid && k < K) {
                    const int ci = k / 9, t = k - 9 * ci, ky = t / 3, kx = t - 3 * ky;
                    if (MODE == 0) {
                        const int y = S * oy + ky - 1, x = S * ox + kx - 1;
                        if (y >= 0 && y < Hl && x >= 0 && x < Wl)
                            v = xin[((int64_t)ci * Hs + (UPS ? (y >> 1) : y)) * Ws + (UPS ? (x >> 1) : x)];
                    } else {
                        const int ty = oy + 1 - ky, tx = ox + 1 - kx;
                        if (ty >= 0 && tx >= 0 && (S == 1 || ((ty & 1) == 0 && (tx & 1) == 0))) {
                            const int gy = ty / S, gx = tx / S;
                            if (gy < Hs && gx < Ws) v = xin[((int64_t)ci * Hs + gy) * Ws + gx];
                        }
                    }
                }
                v2[h] = v;
            }
            packed[q] = pack_bf16x2(v2[0], v2[1]);
        }
        uint8_t *a = sA[stage];
        *reinterpret_cast<uint4 *>(a + kmajor_off(tid, 0)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        *reinterpret_cast<uint4 *>(a + kmajor_off(tid, 8)) = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        // B: the weights of NT channels for these 16 k (zero beyond Cout and K)
        for (int i = tid; i < NT * 16; i += 128) {
            const int n = i >> 4, kk = i & 15, k = kc * 16 + kk;
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (n < Cout && k < K) {
                if (MODE == 0) {
                    v = w[(int64_t)n * K + k];                       // W[co = n][k = (ci, ky, kx)]
                } else {
                    const int co = k / 9, t = k - 9 * co;            // W[co][ci = n][ky, kx]
                    v = w[((int64_t)co * Cout + n) * 9 + t];
                }
            }
            *reinterpret_cast<__nv_bfloat16 *>(sB[stage] + kmajor_off(n, kk)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t ad = umma_desc(smem_u32(sA[stage]), kLBO, kSBO);
            const uint64_t bd = umma_desc(smem_u32(sB[stage]), kLBO, kSBO);
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(kc > 0 ? 1 : 0));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[stage]))
                         : "memory");
        }
        ++issued;
    }
    // the last commit covers every MMA issued before it (also on the error path,
    // before the tensor memory is freed)
    bool done = true;
    if (issued > 0) done = mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
    ok = __syncthreads_and(ok && done) != 0;
    if (!ok && tid == 0) atomicExch(err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // row tid of D: tensor-memory lane 32 * warp + lane, columns 0 .. NT - 1
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (mvalid) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int co = c0 + j;
                    if (co >= Cout) continue;
                    float v = __uint_as_float(r[j]);
                    const int64_t q = ((int64_t)img * Cout + co) * hw + rr;
                    if (MODE == 0) {
                        if (bias) v += bias[co];
                        if (relu) v = fmaxf(v, 0.f);
                        if (out_skip) out_skip[q] = v + skip[q];
                    }
                    out[q] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// Weight gradient of a convolution (MODE 0's layer): with k = (ci, ky, kx),
//   gW[co, k] += sum_{pixels p of this CTA's chunk} X[p][k] g[co, p],
//   X[p][k] = x[n, ci, S oy + ky - 1, S ox + kx - 1] (logical input, upsampled
//   when UPS, zero outside), g = the output gradient [n][Cout][Ho][Wo].
// The contraction runs over pixels: D[m][n] with m = k (128 per CTA: blockIdx.y
// selects the block of k), n = co, K = 16 pixels per MMA, KSTEPS MMAs per CTA
// (blockIdx.x selects the pixel chunk).  Each CTA adds its partial D to gW with
// float atomics.
template <int S, int UPS, int NT, int KSTEPS>
__global__ void __launch_bounds__(128) k_conv_wgrad_tc(const float *__restrict__ x, int Cin, int Hs, int Ws,
                                                       const float *__restrict__ g, int Cout, int Ho, int Wo,
                                                       int64_t npix, float *__restrict__ gw, unsigned *err)
{
    constexpr int TCOLS = NT < 32 ? 32 : NT;
    __shared__ __align__(128) uint8_t sA[2][4096];
    __shared__ __align__(128) uint8_t sB[2][NT * 32];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const int K = Cin * 9;
    const int krow = blockIdx.y * 128 + tid;          // this thread's row of A and of D
    const bool kvalid = krow < K;
    const int ci = kvalid ? krow / 9 : 0, t = krow - 9 * ci, ky = t / 3, kx = t - 3 * ky;
    const int Hl = UPS ? 2 * Hs : Hs, Wl = UPS ? 2 * Ws : Ws;
    const int64_t hw = (int64_t)Ho * Wo;
    const int64_t p0 = (int64_t)blockIdx.x * KSTEPS * 16;
    constexpr uint32_t idesc = umma_idesc_bf16(128, NT);
    bool ok = true;
    int issued = 0;
    for (int kc = 0; kc < KSTEPS; ++kc) {
        const int stage = kc & 1;
        bool free_ok = true;
        if (kc >= 2) free_ok = mbar_wait(&mbar[stage], ((kc - 2) >> 1) & 1);
        ok = __syncthreads_and(free_ok) != 0;
        if (!ok) break;
        // A row krow: X at the 16 pixels of this step
        uint32_t packed[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t p = p0 + kc * 16 + 2 * q + h;
                float v = 0.f;
                if (kvalid && p < npix) {
                    const int img = (int)(p / hw), rr = (int)(p % hw);
                    const int oy = rr / Wo, ox = rr % Wo;
                    const int y = S * oy + ky - 1, xx = S * ox + kx - 1;
                    if (y >= 0 && y < Hl && xx >= 0 && xx < Wl)
                        v = x[(((int64_t)img * Cin + ci) * Hs + (UPS ? (y >> 1) : y)) * Ws + (UPS ? (xx >> 1) : xx)];
                }
                v2[h] = v;
            }
            packed[q] = pack_bf16x2(v2[0], v2[1]);
        }
        uint8_t *a = sA[stage];
        *reinterpret_cast<uint4 *>(a + kmajor_off(tid, 0)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        *reinterpret_cast<uint4 *>(a + kmajor_off(tid, 8)) = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        // B row co: the output gradient at the 16 pixels
        for (int i = tid; i < NT * 16; i += 128) {
            const int n = i >> 4, kk = i & 15;
            const int64_t p = p0 + kc * 16 + kk;
            float v = 0.f;
            if (n < Cout && p < npix) {
                const int img = (int)(p / hw), rr = (int)(p % hw);
                v = g[((int64_t)img * Cout + n) * hw + rr];
            }
            *reinterpret_cast<__nv_bfloat16 *>(sB[stage] + kmajor_off(n, kk)) = __float2bfloat16_rn(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t ad = umma_desc(smem_u32(sA[stage]), kLBO, kSBO);
            const uint64_t bd = umma_desc(smem_u32(sB[stage]), kLBO, kSBO);
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(kc > 0 ? 1 : 0));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[stage]))
                         : "memory");
        }
        ++issued;
    }
    bool done = true;
    if (issued > 0) done = mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
    ok = __syncthreads_and(ok && done) != 0;
    if (!ok && tid == 0) atomicExch(err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (kvalid) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int co = c0 + j;
                    if (co < Cout) atomicAdd(gw + (int64_t)co * K + krow, __uint_as_float(r[j]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

template <int MODE, int S, int UPS>
static void launch_tc(int cout, dim3 grid, cudaStream_t st, const float *in, int Cin, int Hs, int Ws,
                      const __nv_bfloat16 *w, const float *bias, int Ho, int Wo, int relu, const float *skip,
                      float *out, float *out_skip, int64_t npix, unsigned *err)
{
    if (cout <= 16)
        k_conv_tc<MODE, S, UPS, 16><<<grid, 128, 0, st>>>(in, Cin, Hs, Ws, w, bias, cout, Ho, Wo, relu, skip, out,
                                                          out_skip, npix, err);
    else if (cout <= 32)
        k_conv_tc<MODE, S, UPS, 32><<<grid, 128, 0, st>>>(in, Cin, Hs, Ws, w, bias, cout, Ho, Wo, relu, skip, out,
                                                          out_skip, npix, err);
    else
        k_conv_tc<MODE, S, UPS, 64><<<grid, 128, 0, st>>>(in, Cin, Hs, Ws, w, bias, cout, Ho, Wo, relu, skip, out,
                                                          out_skip, npix, err);
}

bool conv_fwd_tc(int S, int UPS, const float *in, int N, int Cin, int Hs, int Ws, const __nv_bfloat16 *w,
                 const float *bias, int Cout, int Ho, int Wo, int relu, const float *skip, float *out,
                 float *out_skip, unsigned *err, cudaStream_t st)
{
    if (Cout < 1 || Cout > 64 || Cin < 1) return false;
    const int64_t npix = (int64_t)N * Ho * Wo;
    const dim3 grid((unsigned)((npix + 127) / 128));
    count_launch();
    if (S == 2 && !UPS) launch_tc<0, 2, 0>(Cout, grid, st, in, Cin, Hs, Ws, w, bias, Ho, Wo, relu, skip, out, out_skip, npix, err);
    else if (S == 1 && UPS) launch_tc<0, 1, 1>(Cout, grid, st, in, Cin, Hs, Ws, w, bias, Ho, Wo, relu, skip, out, out_skip, npix, err);
    else if (S == 1) launch_tc<0, 1, 0>(Cout, grid, st, in, Cin, Hs, Ws, w, bias, Ho, Wo, relu, skip, out, out_skip, npix, err);
    else return false;
    return true;
}

bool conv_bwd_data_tc(int S, const float *gout, int N, int Cout, int Ho, int Wo, const __nv_bfloat16 *w, int Cin,
                      int Hl, int Wl, float *gin, unsigned *err, cudaStream_t st)
{
    if (Cin < 1 || Cin > 64 || Cout < 1) return false;
    const int64_t npix = (int64_t)N * Hl * Wl;
    const dim3 grid((unsigned)((npix + 127) / 128));
    count_launch();
    // the GEMM's K side is the layer's output channels, its N side the input channels
    if (S == 2) launch_tc<1, 2, 0>(Cin, grid, st, gout, Cout, Ho, Wo, w, nullptr, Hl, Wl, 0, nullptr, gin, nullptr, npix, err);
    else if (S == 1) launch_tc<1, 1, 0>(Cin, grid, st, gout, Cout, Ho, Wo, w, nullptr, Hl, Wl, 0, nullptr, gin, nullptr, npix, err);
    else return false;
    return true;
}

// Error word of the stand-alone convolution entry point (mxp_cnn_conv3x3).
static __device__ unsigned g_conv_err;

constexpr int kWgradSteps = 64;        // 16-pixel MMA steps per CTA (1024 pixels)

template <int S, int UPS>
static void launch_wgrad(int cout, dim3 grid, cudaStream_t st, const float *x, int Cin, int Hs, int Ws,
                         const float *g, int Ho, int Wo, int64_t npix, float *gw, unsigned *err)
{
    if (cout <= 16)
        k_conv_wgrad_tc<S, UPS, 16, kWgradSteps><<<grid, 128, 0, st>>>(x, Cin, Hs, Ws, g, cout, Ho, Wo, npix, gw, err);
    else if (cout <= 32)
        k_conv_wgrad_tc<S, UPS, 32, kWgradSteps><<<grid, 128, 0, st>>>(x, Cin, Hs, Ws, g, cout, Ho, Wo, npix, gw, err);
    else
        k_conv_wgrad_tc<S, UPS, 64, kWgradSteps><<<grid, 128, 0, st>>>(x, Cin, Hs, Ws, g, cout, Ho, Wo, npix, gw, err);
}

bool conv_wgrad_tc(int S, int UPS, const float *x, int N, int Cin, int Hs, int Ws, const float *g, int Cout, int Ho,
                   int Wo, float *gw, unsigned *err, cudaStream_t st)
{
    if (Cout < 1 || Cout > 64 || Cin < 1) return false;
    const int64_t npix = (int64_t)N * Ho * Wo;
    const int K = Cin * 9;
    const dim3 grid((unsigned)((npix + kWgradSteps * 16 - 1) / (kWgradSteps * 16)), (unsigned)((K + 127) / 128));
    if (cudaMemsetAsync(gw, 0, (size_t)Cout * K * sizeof(float), st) != cudaSuccess) return false;
    count_launch();
    if (S == 2 && !UPS) launch_wgrad<2, 0>(Cout, grid, st, x, Cin, Hs, Ws, g, Ho, Wo, npix, gw, err);
    else if (S == 1 && UPS) launch_wgrad<1, 1>(Cout, grid, st, x, Cin, Hs, Ws, g, Ho, Wo, npix, gw, err);
    else if (S == 1) launch_wgrad<1, 0>(Cout, grid, st, x, Cin, Hs, Ws, g, Ho, Wo, npix, gw, err);
    else return false;
    return true;
}

}  // namespace mxp

extern "C" mxp_status mxp_cnn_conv3x3(int mode, int stride, int upsample, int N, int Cin, int Hs, int Ws, int Cout,
                                      int Ho, int Wo, const float *a_dev, const float *b_dev,
                                      const void *w_bf16_dev, const float *bias_dev, int relu, float *out_dev,
                                      void *cuda_stream)
{
    using namespace mxp;
    auto bad = [](const char *m) {
        note_error(m);
        return MXP_EINVAL;
    };
    if (mode < 0 || mode > 2) return bad("mode must be 0 (forward), 1 (input gradient) or 2 (weight gradient)");
    if (stride != 1 && stride != 2) return bad("stride must be 1 or 2");
    if (upsample && (stride != 1 || mode == 1)) return bad("upsampling needs stride 1 and mode 0 or 2");
    if (N < 1 || Cin < 1 || Hs < 1 || Ws < 1 || Cout < 1 || Ho < 1 || Wo < 1) return bad("sizes must be >= 1");
    const int Hl = upsample ? 2 * Hs : Hs, Wl = upsample ? 2 * Ws : Ws;
    if (Ho != (Hl + stride - 1) / stride || Wo != (Wl + stride - 1) / stride)
        return bad("Ho, Wo must be the logical input size divided by the stride, rounded up");
    if (!a_dev || !out_dev || (mode != 2 && !w_bf16_dev) || (mode == 2 && !b_dev)) return bad("NULL argument");
    if ((mode == 0 && Cout > 64) || (mode == 1 && Cin > 64) || (mode == 2 && Cout > 64))
        return bad("at most 64 channels on the tensor cores' N side");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_conv_err) != cudaSuccess) {
        note_error("cudaGetSymbolAddress of the error word failed");
        return MXP_ECUDA;
    }
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess) {
        note_error("clearing the error word failed");
        return MXP_ECUDA;
    }
    const __nv_bfloat16 *w = static_cast<const __nv_bfloat16 *>(w_bf16_dev);
    bool ok = false;
    if (mode == 0)
        ok = conv_fwd_tc(stride, upsample, a_dev, N, Cin, Hs, Ws, w, bias_dev, Cout, Ho, Wo, relu, nullptr, out_dev,
                         nullptr, err, st);
    else if (mode == 1)
        ok = conv_bwd_data_tc(stride, a_dev, N, Cout, Ho, Wo, w, Cin, Hs, Ws, out_dev, err, st);
    else
        ok = conv_wgrad_tc(stride, upsample, a_dev, N, Cin, Hs, Ws, b_dev, Cout, Ho, Wo, out_dev, err, st);
    if (!ok) return bad("unsupported convolution shape");
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        note_error(cudaGetErrorString(cudaGetLastError()));
        return MXP_ECUDA;
    }
    if (e) {
        note_error("a tensor-core convolution's bounded wait gave up");
        return MXP_ETIMEOUT;
    }
    return MXP_OK;
}
