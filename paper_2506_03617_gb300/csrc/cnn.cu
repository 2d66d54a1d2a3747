// Learned preconditioning stage: a six-layer U-Net-style CNN with bfloat16
// weights and float32 accumulation, with hand-written forward, backward and
// Adam kernels (training and inference run on the GPU).  The forward
// convolutions, the input gradients and the weight gradients run on the tensor
// cores (tcgen05, bfloat16 operands, float32 accumulation in tensor memory;
// conv_tc.cu); the bias gradients and the elementwise steps on CUDA cores.  The paper has no
// learned stage; this is the project's own extension, used as an extra
// FGMRES stage with MatExPre as fallback (see engine.cu).
//
// Network (NCHW, 3x3 kernels, zero padding 1):
//   a1 = relu(conv(x, W1) + b1)                 3 -> 32
//   a2 = relu(conv_s2(a1, W2) + b2)            32 -> 64, stride 2
//   a3 = relu(conv(a2, W3) + b3)               64 -> 64
//   a4 = relu(conv(a3, W4) + b4)               64 -> 64
//   r5 = relu(conv(up2(a4), W5) + b5), a5 = r5 + a1      64 -> 32, skip
//   y  = conv(a5, W6) + b6                     32 -> 2
// conv_s(x)[o, i, j] = sum_{c, ky, kx} W[o, c, ky, kx] x[c, s i + ky - 1, s j + kx - 1].
// Flat parameters: W1, b1, ..., W6, b6 (W as [c_out][c_in][3][3]).
#include <cmath>
#include <cstring>
#include <vector>

#include "mxp_internal.h"

namespace mxp {

struct CnnLayer {
    int cin, cout, stride, ups, relu;
};
static const CnnLayer kNet[6] = {{3, 32, 1, 0, 1},  {32, 64, 2, 0, 1}, {64, 64, 1, 0, 1},
                                 {64, 64, 1, 0, 1}, {64, 32, 1, 1, 1}, {32, 2, 1, 0, 0}};

static int64_t layer_woff(int l)
{
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)kNet[i].cin * kNet[i].cout * 9 + kNet[i].cout;
    return o;
}
int64_t cnn_num_params() { return layer_woff(6); }

// ---------------------------------------------------------------- backward
// gb[co] = sum over images and pixels of gout[n, co, :, :]; one block per
// channel, fixed-order reduction.
__global__ void __launch_bounds__(256) k_bias_grad(const float *__restrict__ gout, int N, int Cout, int64_t hw,
                                                   float *__restrict__ gb)
{
    const int co = blockIdx.x;
    float acc = 0.f;
    for (int n = 0; n < N; ++n) {
        const float *g = gout + ((int64_t)n * Cout + co) * hw;
        for (int64_t p = threadIdx.x; p < hw; p += blockDim.x) acc += g[p];
    }
    __shared__ float red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int i = 0; i < 8; ++i) v += red[i];
        gb[co] = v;
    }
}

__global__ void k_relu_mask(float *__restrict__ g, const float *__restrict__ a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) g[i] = 0.f;
}

__global__ void k_add_to(float *__restrict__ a, const float *__restrict__ b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// g[n, c, i, j] = sum of the 2 x 2 block of gfull (adjoint of nearest upsampling)
__global__ void k_down2_sum(const float *__restrict__ gfull, int NC, int H, int W, float *__restrict__ g)
{
    const int64_t total = (int64_t)NC * H * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t nc = i / ((int64_t)H * W);
        const int r = (int)(i % ((int64_t)H * W));
        const int y = r / W, x = r % W;
        const float *b = gfull + nc * 4 * H * W;
        const int W2 = 2 * W;
        g[i] = b[(int64_t)(2 * y) * W2 + 2 * x] + b[(int64_t)(2 * y) * W2 + 2 * x + 1] +
               b[(int64_t)(2 * y + 1) * W2 + 2 * x] + b[(int64_t)(2 * y + 1) * W2 + 2 * x + 1];
    }
}

// loss partials and gradient of the mean squared error
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int64_t n,
                      float *__restrict__ gy, double *__restrict__ partial)
{
    double s = 0.0;
    const float sc = 2.0f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        gy[i] = sc * d;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int i = 0; i < (int)(blockDim.x / 32); ++i) v += red[i];
        partial[blockIdx.x] = v;
    }
}

__global__ void k_sum_partials(const double *__restrict__ p, int np, double scale, float *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += p[i];
        *out = (float)(s * scale);
    }
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

// (Re v, Im v, c / c_ref) channels of a 2D grid vector, v scaled by vscale
__global__ void k_pack_input(const double2 *__restrict__ v, const double *__restrict__ c, int64_t n,
                             double vscale, double cscale, float *__restrict__ x)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = (float)(v[i].x * vscale);
        x[n + i] = (float)(v[i].y * vscale);
        x[2 * n + i] = (float)(c[i] * cscale);
    }
}

__global__ void k_unpack_output(const float *__restrict__ y, int64_t n, double2 *__restrict__ z)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = make_double2((double)y[i], (double)y[n + i]);
}

static int ew_grid(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)sm_count() * 8) b = (int64_t)sm_count() * 8;
    return (int)std::max<int64_t>(b, 1);
}

}  // namespace mxp

using namespace mxp;

struct mxp_cnn {
    int device = 0;
    cudaStream_t stream = nullptr;
    int maxn = 0, maxh = 0, maxw = 0;
    int64_t np = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    float *x = nullptr, *a[6] = {nullptr}, *r5 = nullptr, *y = nullptr;
    float *gy = nullptr, *g5 = nullptr, *gfull = nullptr, *gh = nullptr, *gh2 = nullptr, *g1 = nullptr;
    double *partial = nullptr;
    unsigned *err = nullptr;       // set by a tensor-core convolution whose bounded wait gave up
    float *loss_dev = nullptr;
    float *loss_host = nullptr;
    int adam_t = 0;
    int N = 0, H = 0, W = 0;   // shape of the last forward
};

namespace {
mxp_status cfail(mxp_status s, const char *m)
{
    mxp::note_error(m);
    return s;
}
#define CKC(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return cfail(e_ == cudaErrorMemoryAllocation ? MXP_ENOMEM : MXP_ECUDA, \
                                            cudaGetErrorString(e_));                   \
    } while (0)

template <int S, int UPS>
void conv_fwd(const mxp_cnn *net, int l, const float *in, int N, int Hs, int Ws, int Ho, int Wo,
              const float *skip, float *out, float *out_skip)
{
    const CnnLayer L = kNet[l];
    const __nv_bfloat16 *w = net->wb + layer_woff(l);
    const float *b = net->w + layer_woff(l) + (int64_t)L.cin * L.cout * 9;
    conv_fwd_tc(S, UPS, in, N, L.cin, Hs, Ws, w, b, L.cout, Ho, Wo, L.relu, skip, out, out_skip, net->err,
                net->stream);
}

template <int S>
void conv_bwd_data(const mxp_cnn *net, int l, const float *gout, int N, int Ho, int Wo, int Hl, int Wl,
                   float *gin)
{
    const CnnLayer L = kNet[l];
    conv_bwd_data_tc(S, gout, N, L.cout, Ho, Wo, net->wb + layer_woff(l), L.cin, Hl, Wl, gin, net->err,
                     net->stream);
}

template <int S, int UPS>
void conv_bwd_weight(const mxp_cnn *net, int l, const float *xin, int N, int Hs, int Ws, const float *gout,
                     int Ho, int Wo)
{
    const CnnLayer L = kNet[l];
    float *gw = net->g + layer_woff(l);
    float *gb = gw + (int64_t)L.cin * L.cout * 9;
    conv_wgrad_tc(S, UPS, xin, N, L.cin, Hs, Ws, gout, L.cout, Ho, Wo, gw, net->err, net->stream);
    count_launch();
    k_bias_grad<<<L.cout, 256, 0, net->stream>>>(gout, N, L.cout, (int64_t)Ho * Wo, gb);
}

mxp_status check_shape(const mxp_cnn *net, int N, int H, int W)
{
    if (N < 1 || H < 2 || W < 2 || (H & 1) || (W & 1)) return cfail(MXP_EINVAL, "N >= 1 and even H, W >= 2 required");
    if (N > net->maxn || H > net->maxh || W > net->maxw) return cfail(MXP_EINVAL, "shape exceeds the sizes given at creation");
    return MXP_OK;
}

mxp_status forward_impl(mxp_cnn *net, int N, int H, int W, const float *x, float *y)
{
    const int H2 = H / 2, W2 = W / 2;
    conv_fwd<1, 0>(net, 0, x, N, H, W, H, W, nullptr, net->a[0], nullptr);
    conv_fwd<2, 0>(net, 1, net->a[0], N, H, W, H2, W2, nullptr, net->a[1], nullptr);
    conv_fwd<1, 0>(net, 2, net->a[1], N, H2, W2, H2, W2, nullptr, net->a[2], nullptr);
    conv_fwd<1, 0>(net, 3, net->a[2], N, H2, W2, H2, W2, nullptr, net->a[3], nullptr);
    conv_fwd<1, 1>(net, 4, net->a[3], N, H2, W2, H, W, net->a[0], net->r5, net->a[4]);
    conv_fwd<1, 0>(net, 5, net->a[4], N, H, W, H, W, nullptr, y, nullptr);
    net->N = N;
    net->H = H;
    net->W = W;
    CKC(cudaGetLastError());
    return MXP_OK;
}

// parameter gradients of sum(gy * y) for the cached forward, into net->g
mxp_status backward_impl(mxp_cnn *net, const float *x, const float *gy)
{
    const int N = net->N, H = net->H, W = net->W, H2 = H / 2, W2 = W / 2;
    cudaStream_t st = net->stream;
    const int64_t full32 = (int64_t)N * 32 * H * W, half64 = (int64_t)N * 64 * H2 * W2;
    // layer 6
    conv_bwd_weight<1, 0>(net, 5, net->a[4], N, H, W, gy, H, W);
    conv_bwd_data<1>(net, 5, gy, N, H, W, H, W, net->g5);            // d/da5
    // layer 5: a5 = r5 + a1
    CKC(cudaMemcpyAsync(net->g1, net->g5, full32 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    count_launch();
    k_relu_mask<<<ew_grid(full32), 256, 0, st>>>(net->g5, net->r5, full32);
    conv_bwd_weight<1, 1>(net, 4, net->a[3], N, H2, W2, net->g5, H, W);
    conv_bwd_data<1>(net, 4, net->g5, N, H, W, H, W, net->gfull);   // d/d up2(a4), full resolution
    count_launch();
    k_down2_sum<<<ew_grid(half64), 256, 0, st>>>(net->gfull, N * 64, H2, W2, net->gh);
    count_launch();
    k_relu_mask<<<ew_grid(half64), 256, 0, st>>>(net->gh, net->a[3], half64);
    // layer 4
    conv_bwd_weight<1, 0>(net, 3, net->a[2], N, H2, W2, net->gh, H2, W2);
    conv_bwd_data<1>(net, 3, net->gh, N, H2, W2, H2, W2, net->gh2);
    count_launch();
    k_relu_mask<<<ew_grid(half64), 256, 0, st>>>(net->gh2, net->a[2], half64);
    // layer 3
    conv_bwd_weight<1, 0>(net, 2, net->a[1], N, H2, W2, net->gh2, H2, W2);
    conv_bwd_data<1>(net, 2, net->gh2, N, H2, W2, H2, W2, net->gh);
    count_launch();
    k_relu_mask<<<ew_grid(half64), 256, 0, st>>>(net->gh, net->a[1], half64);
    // layer 2 (stride 2)
    conv_bwd_weight<2, 0>(net, 1, net->a[0], N, H, W, net->gh, H2, W2);
    conv_bwd_data<2>(net, 1, net->gh, N, H2, W2, H, W, net->g5);
    count_launch();
    k_add_to<<<ew_grid(full32), 256, 0, st>>>(net->g5, net->g1, full32);
    count_launch();
    k_relu_mask<<<ew_grid(full32), 256, 0, st>>>(net->g5, net->a[0], full32);
    // layer 1
    conv_bwd_weight<1, 0>(net, 0, x, N, H, W, net->g5, H, W);
    CKC(cudaGetLastError());
    return MXP_OK;
}

}  // namespace

extern "C" {

int64_t mxp_cnn_num_params(void) { return cnn_num_params(); }

mxp_status mxp_cnn_create(int device, void *cuda_stream, int max_batch, int max_h, int max_w, mxp_cnn **out)
{
    if (!out) return cfail(MXP_EINVAL, "NULL argument");
    *out = nullptr;
    if (max_batch < 1 || max_h < 2 || max_w < 2 || (max_h & 1) || (max_w & 1))
        return cfail(MXP_EINVAL, "max_batch >= 1 and even max_h, max_w >= 2 required");
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return cfail(MXP_EINVAL, "no such CUDA device");
    mxp_cnn *net = new mxp_cnn();
    net->device = device;
    net->stream = (cudaStream_t)cuda_stream;
    net->maxn = max_batch;
    net->maxh = max_h;
    net->maxw = max_w;
    net->np = cnn_num_params();
    const int64_t N = max_batch, H = max_h, W = max_w;
    const int64_t full = N * H * W, half = N * (H / 2) * (W / 2);
    bool ok = true;
    auto A = [&](void **p, size_t bytes) { ok = ok && cudaMalloc(p, bytes) == cudaSuccess; };
    A((void **)&net->w, net->np * 4); A((void **)&net->g, net->np * 4);
    A((void **)&net->m, net->np * 4); A((void **)&net->v, net->np * 4);
    A((void **)&net->wb, net->np * 2);
    A((void **)&net->x, full * 3 * 4);
    A((void **)&net->a[0], full * 32 * 4); A((void **)&net->a[1], half * 64 * 4);
    A((void **)&net->a[2], half * 64 * 4); A((void **)&net->a[3], half * 64 * 4);
    A((void **)&net->a[4], full * 32 * 4); A((void **)&net->r5, full * 32 * 4);
    A((void **)&net->y, full * 2 * 4); A((void **)&net->gy, full * 2 * 4);
    A((void **)&net->g5, full * 32 * 4); A((void **)&net->g1, full * 32 * 4);
    A((void **)&net->gfull, full * 64 * 4); A((void **)&net->gh, half * 64 * 4);
    A((void **)&net->gh2, half * 64 * 4);
    A((void **)&net->partial, 2048 * sizeof(double)); A((void **)&net->loss_dev, sizeof(float));
    A((void **)&net->err, sizeof(unsigned));
    ok = ok && cudaMallocHost((void **)&net->loss_host, sizeof(float)) == cudaSuccess;
    if (ok) {
        ok = cudaMemsetAsync(net->w, 0, net->np * 4, net->stream) == cudaSuccess &&
             cudaMemsetAsync(net->m, 0, net->np * 4, net->stream) == cudaSuccess &&
             cudaMemsetAsync(net->v, 0, net->np * 4, net->stream) == cudaSuccess &&
             cudaMemsetAsync(net->wb, 0, net->np * 2, net->stream) == cudaSuccess &&
             cudaMemsetAsync(net->err, 0, sizeof(unsigned), net->stream) == cudaSuccess &&
             cudaStreamSynchronize(net->stream) == cudaSuccess;
    }
    cudaSetDevice(prev);
    if (!ok) {
        mxp_cnn_destroy(net);
        return cfail(MXP_ENOMEM, "allocation of the network buffers failed");
    }
    *out = net;
    return MXP_OK;
}

mxp_status mxp_cnn_set_params(mxp_cnn *net, const float *host_params)
{
    if (!net || !host_params) return cfail(MXP_EINVAL, "NULL argument");
    for (int64_t i = 0; i < net->np; ++i)
        if (!std::isfinite(host_params[i])) return cfail(MXP_EINVAL, "parameters must be finite");
    CKC(cudaMemcpyAsync(net->w, host_params, net->np * 4, cudaMemcpyHostToDevice, net->stream));
    CKC(cudaMemsetAsync(net->m, 0, net->np * 4, net->stream));
    CKC(cudaMemsetAsync(net->v, 0, net->np * 4, net->stream));
    count_launch();
    k_to_bf16<<<ew_grid(net->np), 256, 0, net->stream>>>(net->w, net->wb, net->np);
    CKC(cudaStreamSynchronize(net->stream));
    net->adam_t = 0;
    return MXP_OK;
}

mxp_status mxp_cnn_get_params(const mxp_cnn *net, float *host_params)
{
    if (!net || !host_params) return cfail(MXP_EINVAL, "NULL argument");
    CKC(cudaMemcpyAsync(host_params, net->w, net->np * 4, cudaMemcpyDeviceToHost, net->stream));
    CKC(cudaStreamSynchronize(net->stream));
    return MXP_OK;
}

// Reads (and clears) the tensor-core error word; one stream synchronisation.
static mxp_status check_tc_error(mxp_cnn *net)
{
    unsigned e = 0;
    CKC(cudaMemcpyAsync(&e, net->err, sizeof(unsigned), cudaMemcpyDeviceToHost, net->stream));
    CKC(cudaStreamSynchronize(net->stream));
    if (e) {
        CKC(cudaMemsetAsync(net->err, 0, sizeof(unsigned), net->stream));
        return cfail(MXP_ETIMEOUT, "a tensor-core convolution's bounded wait gave up");
    }
    return MXP_OK;
}

mxp_status mxp_cnn_forward(mxp_cnn *net, int N, int H, int W, const float *x_dev, float *y_dev)
{
    if (!net || !x_dev || !y_dev) return cfail(MXP_EINVAL, "NULL argument");
    mxp_status s = check_shape(net, N, H, W);
    if (s != MXP_OK) return s;
    s = forward_impl(net, N, H, W, x_dev, y_dev);
    if (s != MXP_OK) return s;
    return check_tc_error(net);
}

mxp_status mxp_cnn_backward(mxp_cnn *net, const float *x_dev, const float *gy_dev, float *grad_dev)
{
    if (!net || !x_dev || !gy_dev || !grad_dev) return cfail(MXP_EINVAL, "NULL argument");
    if (net->N == 0) return cfail(MXP_EINVAL, "backward needs a preceding forward");
    mxp_status s = backward_impl(net, x_dev, gy_dev);
    if (s != MXP_OK) return s;
    CKC(cudaMemcpyAsync(grad_dev, net->g, net->np * 4, cudaMemcpyDeviceToDevice, net->stream));
    return MXP_OK;
}

mxp_status mxp_cnn_train_step(mxp_cnn *net, int N, int H, int W, const float *x_dev, const float *target_dev,
                              float lr, float *loss_out)
{
    if (!net || !x_dev || !target_dev) return cfail(MXP_EINVAL, "NULL argument");
    if (!(lr > 0) || !std::isfinite(lr)) return cfail(MXP_EINVAL, "lr must be finite and > 0");
    mxp_status s = check_shape(net, N, H, W);
    if (s != MXP_OK) return s;
    s = forward_impl(net, N, H, W, x_dev, net->y);
    if (s != MXP_OK) return s;
    const int64_t ny = (int64_t)N * 2 * H * W;
    const int nb = std::min(ew_grid(ny), 2048);
    count_launch(2);
    k_mse<<<nb, 256, 0, net->stream>>>(net->y, target_dev, ny, net->gy, net->partial);
    k_sum_partials<<<1, 32, 0, net->stream>>>(net->partial, nb, 1.0 / (double)ny, net->loss_dev);
    s = backward_impl(net, x_dev, net->gy);
    if (s != MXP_OK) return s;
    net->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->adam_t), c2 = 1.f - std::pow(b2, (float)net->adam_t);
    count_launch();
    k_adam<<<ew_grid(net->np), 256, 0, net->stream>>>(net->w, net->g, net->m, net->v, net->wb, net->np, lr, b1,
                                                     b2, 1e-8f, c1, c2);
    CKC(cudaGetLastError());
    if (loss_out) {
        CKC(cudaMemcpyAsync(net->loss_host, net->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, net->stream));
        s = check_tc_error(net);
        if (s != MXP_OK) return s;
        *loss_out = *net->loss_host;
        if (!std::isfinite(*loss_out)) return cfail(MXP_ENAN, "training loss is not finite");
    }
    return MXP_OK;
}

void mxp_cnn_destroy(mxp_cnn *net)
{
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    float *bufs[] = {net->w, net->g, net->m, net->v, net->x, net->a[0], net->a[1], net->a[2], net->a[3],
                     net->a[4], net->r5, net->y, net->gy, net->g5, net->g1, net->gfull, net->gh, net->gh2,
                     net->loss_dev};
    for (float *b : bufs) cudaFree(b);
    cudaFree(net->wb);
    cudaFree(net->err);
    cudaFree(net->partial);
    if (net->loss_host) cudaFreeHost(net->loss_host);
    delete net;
}

}  // extern "C"

// z = network(v) for the learned FGMRES stage: inputs (Re v, Im v, c / c_max)
// with v scaled to unit root-mean-square; output channels (Re z, Im z).
mxp_status mxp::cnn_apply_vector(mxp_cnn *net, int n0, int n1, const double2 *v, double vnorm,
                                 const double *c, double cmax, double2 *z)
{
    mxp_status s = check_shape(net, 1, n1, n0);
    if (s != MXP_OK) return s;
    const int64_t n = (int64_t)n0 * n1;
    const double vscale = vnorm > 0 ? std::sqrt((double)n) / vnorm : 0.0;
    count_launch();
    k_pack_input<<<ew_grid(n), 256, 0, net->stream>>>(v, c, n, vscale, 1.0 / cmax, net->x);
    s = forward_impl(net, 1, n1, n0, net->x, net->y);
    if (s != MXP_OK) return s;
    count_launch();
    k_unpack_output<<<ew_grid(n), 256, 0, net->stream>>>(net->y, n, z);
    CKC(cudaGetLastError());
    return check_tc_error(net);
}
