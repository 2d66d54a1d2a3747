// Stencil kernels: the PML Helmholtz operator and one Taylor-Horner step of the
// exponential-integrator actions (Def. psi), for complex128, complex64 and
// bfloat16-storage vectors.
//
// Operator (Eq. helmholtz with the stretched Laplacian of Eq. pml-1d-s on each
// axis, shift of Sec. 3.4), written with the per-axis coefficient table
//   wp_d[i] = a_d(i) b_d(i+1/2) / h^2,  wm_d[i] = a_d(i) b_d(i-1/2) / h^2,
//   wc_d[i] = wp_d[i] + wm_d[i]   (a, b = 1/s at nodes and half nodes):
//   (A_s p)_q = sum_d (wp_d p_{q+e_d} + wm_d p_{q-e_d} - wc_d p_q)
//               + kappa_q (1 + i s) p_q,          kappa = omega^2 / c^2,
// with p = 0 outside the grid (Dirichlet).
#include "mxp_internal.h"

namespace mxp {

int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            return 152;
        }
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <typename C>
__device__ __forceinline__ C czero() { return CT<C>::mk(0, 0); }

// out = rho * ( y + sigma * ((A_s - mu) p) + gamma * v )
// HAS_Y = false drops y; HAS_V = false drops v.
template <typename S, int DIM, bool HAS_Y, bool HAS_V>
__global__ void __launch_bounds__(128) k_step(Geom g, const typename St<S>::C *__restrict__ coef,
                                              const typename St<S>::R *__restrict__ kappa,
                                              StepScalars<typename St<S>::C> sc,
                                              const S *__restrict__ pin, const S *__restrict__ y,
                                              const S *__restrict__ v, S *__restrict__ pout)
{
    using C = typename St<S>::C;
    using R = typename St<S>::R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int k = blockIdx.z;
    if (i >= g.n[0]) return;
    const int64_t q = i + g.s1 * j + g.s2 * k;
    const int nm = g.nmax;
    const C pc = St<S>::ld(pin, q);
    C acc = czero<C>();
    C wcs = czero<C>();
    // outside the PML every neighbour coefficient is the real 1/h^2: add the
    // neighbours and scale once instead of multiplying complex coefficients
    const int p0 = g.npml;
    const bool inner = g.fast && i >= p0 && i < g.n[0] - p0 && (DIM < 2 || (j >= p0 && j < g.n[1] - p0)) &&
                       (DIM < 3 || (k >= p0 && k < g.n[2] - p0));
    {
        const C xp = (i + 1 < g.n[0]) ? St<S>::ld(pin, q + 1) : czero<C>();
        const C xm = (i > 0) ? St<S>::ld(pin, q - 1) : czero<C>();
        acc = inner ? cadd(xp, xm) : cadd(cmul(coef[i], xp), cmul(coef[nm + i], xm));
        wcs = cadd(wcs, coef[2 * nm + i]);
    }
    if (DIM >= 2) {
        const C *cf = coef + 3 * nm;
        const C xp = (j + 1 < g.n[1]) ? St<S>::ld(pin, q + g.s1) : czero<C>();
        const C xm = (j > 0) ? St<S>::ld(pin, q - g.s1) : czero<C>();
        acc = cadd(acc, inner ? cadd(xp, xm) : cadd(cmul(cf[j], xp), cmul(cf[nm + j], xm)));
        wcs = cadd(wcs, cf[2 * nm + j]);
    }
    if (DIM >= 3) {
        const C *cf = coef + 6 * nm;
        const C xp = (k + 1 < g.n[2]) ? St<S>::ld(pin, q + g.s2) : czero<C>();
        const C xm = (k > 0) ? St<S>::ld(pin, q - g.s2) : czero<C>();
        acc = cadd(acc, inner ? cadd(xp, xm) : cadd(cmul(cf[k], xp), cmul(cf[nm + k], xm)));
        wcs = cadd(wcs, cf[2 * nm + k]);
    }
    if (inner) {
        const R s = (R)g.ih2;
        acc = CT<C>::mk(acc.x * s, acc.y * s);
    }
    const R kp = kappa[q];
    // diagonal: kappa (1 + i s) - mu - sum_d wc_d
    C diag = CT<C>::mk(kp * sc.zfac.x - sc.mu - wcs.x, kp * sc.zfac.y - wcs.y);
    if (sc.nfaces) {
        // rows on a sound-hard or absorbing face: the ghost value is a multiple of
        // the row's own unknown, so its coefficient joins the diagonal
        const int n0 = g.n[0], n1 = g.n[1];
        if (sc.face[0] && i == 0) diag = cadd(diag, sc.face[0][j + (int64_t)n1 * k]);
        if (sc.face[1] && i == n0 - 1) diag = cadd(diag, sc.face[1][j + (int64_t)n1 * k]);
        if (DIM >= 2) {
            if (sc.face[2] && j == 0) diag = cadd(diag, sc.face[2][i + (int64_t)n0 * k]);
            if (sc.face[3] && j == n1 - 1) diag = cadd(diag, sc.face[3][i + (int64_t)n0 * k]);
        }
        if (DIM >= 3) {
            if (sc.face[4] && k == 0) diag = cadd(diag, sc.face[4][i + (int64_t)n0 * j]);
            if (sc.face[5] && k == g.n[2] - 1) diag = cadd(diag, sc.face[5][i + (int64_t)n0 * j]);
        }
    }
    acc = cadd(acc, cmul(diag, pc));
    C out = cmul(sc.sigma, acc);
    if (HAS_Y) out = cadd(out, St<S>::ld(y, q));
    if (HAS_V) out = cadd(out, cmul(sc.gamma, St<S>::ld(v, q)));
    out = cmul(sc.rho, out);
    St<S>::st(pout, q, out);
}

// The same Taylor-Horner step on a 3D grid, marching along z: a thread owns
// one (x, y) column over a segment of LZ planes and keeps p at z-1, z and z+1 in
// registers, so a point reads only the next plane of p from memory; its x and y
// neighbours lie in the plane the neighbouring threads of the block load at the
// same step (L1 hits).  DRAM traffic is then the compulsory p, y, kappa reads and
// the p write of every point, plus two planes per segment.  Zero Dirichlet faces
// only (faces with ghost terms use k_step).
template <typename S, bool HAS_Y, bool HAS_V>
__global__ void __launch_bounds__(256) k_step3z(Geom g, const typename St<S>::C *__restrict__ coef,
                                                const typename St<S>::R *__restrict__ kappa,
                                                StepScalars<typename St<S>::C> sc,
                                                const S *__restrict__ pin, const S *__restrict__ y,
                                                const S *__restrict__ v, S *__restrict__ pout, int lz)
{
    using C = typename St<S>::C;
    using R = typename St<S>::R;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], nm = g.nmax;
    if (i >= n0 || j >= n1) return;
    const int z0 = blockIdx.z * lz;
    const int z1 = min(z0 + lz, n2);
    const int p0 = g.npml;
    const bool xyin = g.fast && i >= p0 && i < n0 - p0 && j >= p0 && j < n1 - p0;
    const C wpx = coef[i], wmx = coef[nm + i], wcx = coef[2 * nm + i];
    const C wpy = coef[3 * nm + j], wmy = coef[4 * nm + j], wcy = coef[5 * nm + j];
    const C *cz = coef + 6 * nm;
    int64_t q = i + g.s1 * j + g.s2 * z0;
    C pm = (z0 > 0) ? St<S>::ld(pin, q - g.s2) : czero<C>();
    C pc = St<S>::ld(pin, q);
    for (int k = z0; k < z1; ++k, q += g.s2) {
        const C pp = (k + 1 < n2) ? St<S>::ld(pin, q + g.s2) : czero<C>();
        const C xp = (i + 1 < n0) ? St<S>::ld(pin, q + 1) : czero<C>();
        const C xm = (i > 0) ? St<S>::ld(pin, q - 1) : czero<C>();
        const C yp = (j + 1 < n1) ? St<S>::ld(pin, q + g.s1) : czero<C>();
        const C ym = (j > 0) ? St<S>::ld(pin, q - g.s1) : czero<C>();
        const bool inner = xyin && k >= p0 && k < n2 - p0;
        C acc;
        if (inner) {
            acc = cadd(cadd(cadd(xp, xm), cadd(yp, ym)), cadd(pp, pm));
            const R s = (R)g.ih2;
            acc = CT<C>::mk(acc.x * s, acc.y * s);
        } else {
            acc = cadd(cmul(wpx, xp), cmul(wmx, xm));
            acc = cadd(acc, cadd(cmul(wpy, yp), cmul(wmy, ym)));
            acc = cadd(acc, cadd(cmul(cz[k], pp), cmul(cz[nm + k], pm)));
        }
        const C wcs = cadd(cadd(wcx, wcy), cz[2 * nm + k]);
        const R kp = kappa[q];
        const C diag = CT<C>::mk(kp * sc.zfac.x - sc.mu - wcs.x, kp * sc.zfac.y - wcs.y);
        acc = cadd(acc, cmul(diag, pc));
        C out = cmul(sc.sigma, acc);
        if (HAS_Y) out = cadd(out, St<S>::ld(y, q));
        if (HAS_V) out = cadd(out, cmul(sc.gamma, St<S>::ld(v, q)));
        out = cmul(sc.rho, out);
        St<S>::st(pout, q, out);
        pm = pc;
        pc = pp;
    }
}

// Planes per z segment: enough segments for about four waves of 256-thread
// blocks at eight blocks per SM, at least four planes each.
static int z_segment(const Geom &g)
{
    const int64_t bxy = (int64_t)((g.n[0] + 31) / 32) * ((g.n[1] + 7) / 8);
    const int64_t want = (int64_t)sm_count() * 8 * 4;
    int64_t nseg = (want + bxy - 1) / bxy;
    if (nseg < 1) nseg = 1;
    int lz = (int)((g.n[2] + nseg - 1) / nseg);
    if (lz < 4) lz = 4;
    return lz;
}

template <typename S>
static void launch_step3z(const Geom &g, const typename St<S>::C *coef, const typename St<S>::R *kappa,
                          const StepScalars<typename St<S>::C> &sc, const S *pin, const S *y,
                          const S *v, S *pout, cudaStream_t st)
{
    const int lz = z_segment(g);
    dim3 block(32, 8);
    dim3 grid((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + lz - 1) / lz);
    count_launch();
    if (y && v) k_step3z<S, true, true><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout, lz);
    else if (y) k_step3z<S, true, false><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout, lz);
    else if (v) k_step3z<S, false, true><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout, lz);
    else k_step3z<S, false, false><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout, lz);
}

template <typename S, int DIM>
static void launch_step_dim(const Geom &g, const typename St<S>::C *coef,
                            const typename St<S>::R *kappa,
                            const StepScalars<typename St<S>::C> &sc, const S *pin, const S *y,
                            const S *v, S *pout, cudaStream_t st)
{
    dim3 block(128);
    dim3 grid((g.n[0] + 127) / 128, g.n[1], g.n[2]);
    count_launch();
    if (y && v) k_step<S, DIM, true, true><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout);
    else if (y) k_step<S, DIM, true, false><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout);
    else if (v) k_step<S, DIM, false, true><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout);
    else k_step<S, DIM, false, false><<<grid, block, 0, st>>>(g, coef, kappa, sc, pin, y, v, pout);
}

template <typename S>
void launch_step(const Geom &g, const typename St<S>::C *coef, const typename St<S>::R *kappa,
                 const StepScalars<typename St<S>::C> &sc, const S *pin, const S *y, const S *v,
                 S *pout, cudaStream_t st)
{
    if constexpr (sizeof(S) <= 8) {                                      // complex64 / bf16 storage
        if (g.dim == 3 && sc.nfaces == 0) {
            launch_step3z<S>(g, coef, kappa, sc, pin, y, v, pout, st);
            return;
        }
    }
    if (g.dim == 3) launch_step_dim<S, 3>(g, coef, kappa, sc, pin, y, v, pout, st);
    else launch_step_dim<S, 2>(g, coef, kappa, sc, pin, y, v, pout, st);
}

// ---------------------------------------------------------------- conversions
template <typename S>
__global__ void k_convert_in(const double2 *__restrict__ x, S *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        St<S>::st(out, i, St<S>::from64(x[i]));
}

template <typename S>
__global__ void k_convert_out(const S *__restrict__ x, double2 *__restrict__ out,
                              const double2 *__restrict__ base, int mode, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const auto c = St<S>::ld(x, i);
        double2 r = make_double2((double)c.x, (double)c.y);
        if (mode == 1) r = csub(base[i], r);
        out[i] = r;
    }
}

static int stream_grid(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)sm_count() * 16) b = (int64_t)sm_count() * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename S>
void launch_convert_in(const double2 *x, S *out, int64_t n, cudaStream_t st)
{
    count_launch();
    k_convert_in<S><<<stream_grid(n), 256, 0, st>>>(x, out, n);
}

template <typename S>
void launch_convert_out(const S *x, double2 *out, const double2 *base, int mode, int64_t n,
                        cudaStream_t st)
{
    count_launch();
    k_convert_out<S><<<stream_grid(n), 256, 0, st>>>(x, out, base, mode, n);
}

#define MXP_INST(S)                                                                          \
    template void launch_step<S>(const Geom &, const St<S>::C *, const St<S>::R *,           \
                                 const StepScalars<St<S>::C> &, const S *, const S *,        \
                                 const S *, S *, cudaStream_t);                              \
    template void launch_convert_in<S>(const double2 *, S *, int64_t, cudaStream_t);         \
    template void launch_convert_out<S>(const S *, double2 *, const double2 *, int, int64_t, \
                                        cudaStream_t);
MXP_INST(double2)
MXP_INST(float2)
MXP_INST(__nv_bfloat162)
#undef MXP_INST

}  // namespace mxp
