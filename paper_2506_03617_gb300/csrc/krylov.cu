// Krylov vector kernels in complex128 / FP64 for the inner GMRES of Algorithm 1
// and the outer FGMRES (Sec. 3.4): blocked multi-dot products with a fixed-order
// two-stage reduction (bitwise reproducible for a given grid size), multi-axpy,
// norms, and the Hessenberg / Givens least-squares update kept on the device.
#include "mxp_internal.h"

namespace mxp {

std::atomic<long long> g_launch_count{0};

constexpr int kRedThreads = 256;

__device__ __forceinline__ double2 warp_sum(double2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Block b writes partials[b * kChunk + i] = sum over its points of conj(V_i) w.
// A launch with gate != nullptr does nothing unless *gate != 0 (device-side
// decision of the selective second Gram-Schmidt pass).
template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_mdot_partial(const double2 *__restrict__ V,
                                                              int64_t ld,
                                                              const double2 *__restrict__ w,
                                                              int64_t n,
                                                              double2 *__restrict__ partials,
                                                              const double *__restrict__ gate)
{
    if (gate && *gate == 0.0) return;
    double2 acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = make_double2(0.0, 0.0);
    for (int64_t p = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kRedThreads) {
        const double2 wp = w[p];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const double2 a = V[v * ld + p];
            acc[v].x += a.x * wp.x + a.y * wp.y;   // conj(a) * w
            acc[v].y += a.x * wp.y - a.y * wp.x;
        }
    }
    __shared__ double2 red[kRedThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double2 s = warp_sum(acc[v]);
        if (lane == 0) red[warp][v] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double2 s = make_double2(0.0, 0.0);
        for (int wi = 0; wi < kRedThreads / 32; ++wi) s = cadd(s, red[wi][threadIdx.x]);
        partials[blockIdx.x * kChunk + threadIdx.x] = s;
    }
}

// out[i] (+)= sum_b partials[b * kChunk + i], b in fixed order; one warp per i.
__global__ void k_reduce_partials(const double2 *__restrict__ partials, int nblocks, int nv,
                                  double2 *__restrict__ out, int accumulate,
                                  const double *__restrict__ gate)
{
    if (gate && *gate == 0.0) return;
    const int i = blockIdx.x;
    if (i >= nv) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nblocks; b += 32) s = cadd(s, partials[b * kChunk + i]);
    s = warp_sum(s);
    if (threadIdx.x == 0) out[i] = accumulate ? cadd(out[i], s) : s;
}

void krylov_mdot(const double2 *V, int64_t ld, int nvec, const double2 *w, int64_t n,
                 double2 *out, int accumulate, const KrylovScratch &ks, cudaStream_t st,
                 const double *gate)
{
    for (int base = 0; base < nvec; base += kChunk) {
        const int nv = (nvec - base < kChunk) ? nvec - base : kChunk;
        const double2 *Vb = V + base * ld;
        switch (nv) {
#define MXP_CASE(NVV) \
    case NVV: count_launch(); k_mdot_partial<NVV><<<ks.grid, kRedThreads, 0, st>>>(Vb, ld, w, n, ks.partials, gate); break;
            MXP_CASE(1) MXP_CASE(2) MXP_CASE(3) MXP_CASE(4)
            MXP_CASE(5) MXP_CASE(6) MXP_CASE(7) MXP_CASE(8)
#undef MXP_CASE
        }
        count_launch();
        k_reduce_partials<<<nv, 32, 0, st>>>(ks.partials, ks.grid, nv, out + base, accumulate, gate);
    }
}

// w += sign * sum_i coef[i] V_i
__global__ void k_maxpy(double2 *__restrict__ w, const double2 *__restrict__ V, int64_t ld,
                        int nvec, const double2 *__restrict__ coef, double sign, int64_t n,
                        const double *__restrict__ gate)
{
    if (gate && *gate == 0.0) return;
    __shared__ double2 cf[64];
    for (int i = threadIdx.x; i < nvec; i += blockDim.x)
        cf[i] = make_double2(sign * coef[i].x, sign * coef[i].y);
    __syncthreads();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = w[p];
        for (int i = 0; i < nvec; ++i) acc = cadd(acc, cmul(cf[i], V[i * ld + p]));
        w[p] = acc;
    }
}

static int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > (int64_t)sm_count() * 8) b = (int64_t)sm_count() * 8;
    if (b < 1) b = 1;
    return (int)b;
}

void krylov_maxpy(double2 *w, const double2 *V, int64_t ld, int nvec, const double2 *coef,
                  double sign, int64_t n, cudaStream_t st, const double *gate)
{
    if (nvec <= 0) return;
    count_launch();
    k_maxpy<<<grid_for(n, 256), 256, 0, st>>>(w, V, ld, nvec, coef, sign, n, gate);
}

__global__ void k_nrm_partial(const double2 *__restrict__ w, int64_t n, double2 *__restrict__ partials)
{
    double s = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kRedThreads) {
        const double2 a = w[p];
        s += a.x * a.x + a.y * a.y;
    }
    double2 v = warp_sum(make_double2(s, 0.0));
    __shared__ double red[kRedThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRedThreads / 32; ++i) t += red[i];
        partials[blockIdx.x * kChunk] = make_double2(t, 0.0);
    }
}

__global__ void k_reduce_real(const double2 *__restrict__ partials, int nblocks, double *out)
{
    double2 s = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nblocks; b += 32) s.x += partials[b * kChunk].x;
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = s.x;
}

void krylov_nrm2sq(const double2 *w, int64_t n, double *out_dev, const KrylovScratch &ks,
                   cudaStream_t st)
{
    count_launch();
    k_nrm_partial<<<ks.grid, kRedThreads, 0, st>>>(w, n, ks.partials);
    count_launch();
    k_reduce_real<<<1, 32, 0, st>>>(ks.partials, ks.grid, out_dev);
}

__global__ void k_scale_invnorm(double2 *__restrict__ w, const double2 *__restrict__ x,
                                const double *__restrict__ nrm2sq, int64_t n)
{
    const double s2 = *nrm2sq;
    const double inv = (s2 > 0.0) ? 1.0 / sqrt(s2) : 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = x[p];
        w[p] = make_double2(a.x * inv, a.y * inv);
    }
}

void krylov_scale_invnorm(double2 *w, const double2 *x, const double *nrm2sq_dev, int64_t n,
                          cudaStream_t st)
{
    count_launch();
    k_scale_invnorm<<<grid_for(n, 256), 256, 0, st>>>(w, x, nrm2sq_dev, n);
}

__global__ void k_sub(double2 *out, const double2 *a, const double2 *b, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = csub(a[p], b[p]);
}

void krylov_sub(double2 *out, const double2 *a, const double2 *b, int64_t n, cudaStream_t st)
{
    count_launch();
    k_sub<<<grid_for(n, 256), 256, 0, st>>>(out, a, b, n);
}

__global__ void k_add(double2 *out, const double2 *a, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = cadd(out[p], a[p]);
}

void krylov_add(double2 *out, const double2 *a, int64_t n, cudaStream_t st)
{
    count_launch();
    k_add<<<grid_for(n, 256), 256, 0, st>>>(out, a, n);
}

__global__ void k_scale(double2 *__restrict__ w, double2 a, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = w[p];
        w[p] = make_double2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
    }
}

void krylov_scale(double2 *w, double2 a, int64_t n, cudaStream_t st)
{
    count_launch();
    k_scale<<<grid_for(n, 256), 256, 0, st>>>(w, a, n);
}

void krylov_copy(double2 *out, const double2 *a, int64_t n, cudaStream_t st)
{
    cudaMemcpyAsync(out, a, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
}

// ---------------------------------------------------------------- Hessenberg
// Complex Givens rotation [c s; -conj(s) c] that zeroes b in (a, b).
__device__ void givens_make(double2 a, double2 b, double *c, double2 *s)
{
    const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
    if (nb == 0.0) { *c = 1.0; *s = make_double2(0.0, 0.0); return; }
    if (na == 0.0) { *c = 0.0; *s = make_double2(b.x / nb, -b.y / nb); return; }
    const double r = hypot(na, nb);
    *c = na / r;
    const double2 ua = make_double2(a.x / na, a.y / na);       // a / |a|
    const double2 cb = make_double2(b.x / r, -b.y / r);         // conj(b) / r
    *s = cmul(ua, cb);
}

__global__ void k_hess_update(double2 *H, double *cs, double2 *sn, double2 *g, double *scal,
                              int j, int R)
{
    double2 *col = H + (size_t)j * (R + 1);
    const double hn = sqrt(scal[0]);
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], b = col[i + 1];
        const double c = cs[i];
        const double2 s = sn[i];
        col[i] = cadd(make_double2(c * a.x, c * a.y), cmul(s, b));
        const double2 sc = make_double2(-s.x, s.y);               // -conj(s)
        col[i + 1] = cadd(cmul(sc, a), make_double2(c * b.x, c * b.y));
    }
    double c;
    double2 s;
    givens_make(col[j], col[j + 1], &c, &s);
    const double2 a = col[j], b = col[j + 1];
    col[j] = cadd(make_double2(c * a.x, c * a.y), cmul(s, b));
    col[j + 1] = make_double2(0.0, 0.0);
    cs[j] = c;
    sn[j] = s;
    const double2 gj = g[j];
    g[j + 1] = cmul(make_double2(-s.x, s.y), gj);
    g[j] = make_double2(c * gj.x, c * gj.y);
    scal[1] = hypot(g[j + 1].x, g[j + 1].y);
    scal[2] = (hn == 0.0) ? 1.0 : 0.0;
}

void hess_update(const HessState &hs, int j, cudaStream_t st)
{
    count_launch();
    k_hess_update<<<1, 1, 0, st>>>(hs.H, hs.cs, hs.sn, hs.g, hs.scal, j, hs.R);
}

__global__ void k_hess_start(double2 *g, double *scal, int R)
{
    const double beta = sqrt(scal[0]);
    g[0] = make_double2(beta, 0.0);
    for (int i = 1; i <= R; ++i) g[i] = make_double2(0.0, 0.0);
    scal[1] = beta;
    scal[2] = 0.0;
    scal[3] = beta;
}

void hess_start(const HessState &hs, cudaStream_t st)
{
    count_launch();
    k_hess_start<<<1, 1, 0, st>>>(hs.g, hs.scal, hs.R);
}

__device__ double2 cdiv(double2 a, double2 b)
{
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__global__ void k_hess_backsolve(const double2 *H, const double2 *g, double2 *y, int j, int R)
{
    for (int i = j - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int k = i + 1; k < j; ++k) s = csub(s, cmul(H[(size_t)k * (R + 1) + i], y[k]));
        y[i] = cdiv(s, H[(size_t)i * (R + 1) + i]);
    }
}

void hess_backsolve(const HessState &hs, int j, cudaStream_t st)
{
    count_launch();
    k_hess_backsolve<<<1, 1, 0, st>>>(hs.H, hs.g, hs.y, j, hs.R);
}

__global__ void k_addvec(double2 *a, const double2 *b, int n, const double *__restrict__ gate)
{
    if (gate && *gate == 0.0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = cadd(a[i], b[i]);
}

void krylov_addvec(double2 *a, const double2 *b, int n, cudaStream_t st, const double *gate)
{
    count_launch();
    k_addvec<<<(n + 63) / 64, 64, 0, st>>>(a, b, n, gate);
}

// Is a second classical Gram-Schmidt pass needed?  col[0..j] holds the first
// pass's projections h_i and col[j+1].x the squared norm of w before them, so
// ||w - V h||^2 = ||w||^2 - sum |h_i|^2 in exact arithmetic.  The pass is
// repeated when the part of w left after the first pass is below eta ||w||
// (the "twice is enough" test); the estimate only errs towards repeating.
constexpr double kReorthEta2 = 0.01;   // eta^2, eta = 0.1
__global__ void k_reorth_gate(const double2 *__restrict__ col, int j, double *__restrict__ gate)
{
    const double nw = col[j + 1].x;
    double proj = 0.0;
    for (int i = 0; i <= j; ++i) proj += col[i].x * col[i].x + col[i].y * col[i].y;
    *gate = (nw - proj < kReorthEta2 * nw) ? 1.0 : 0.0;
}

void krylov_reorth_gate(const double2 *col, int j, double *gate, cudaStream_t st)
{
    count_launch();
    k_reorth_gate<<<1, 1, 0, st>>>(col, j, gate);
}

__global__ void k_kappa(const double *__restrict__ c, double w2, double *__restrict__ k64,
                        float *__restrict__ k32, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double v = w2 / (c[p] * c[p]);
        k64[p] = v;
        k32[p] = (float)v;
    }
}

void compute_kappa(const double *c, double omega, double *k64, float *k32, int64_t n,
                   cudaStream_t st)
{
    count_launch();
    k_kappa<<<grid_for(n, 256), 256, 0, st>>>(c, omega * omega, k64, k32, n);
}

}  // namespace mxp
