// Allocation-free exp / psi_1 action (mxp_apply_phi_noalloc).
//
// Some callers cannot allocate device memory at the point where they need an
// action: plugins whose host application owns every byte of device memory
// through its own pool, and loops where a cudaMalloc (which may synchronise the
// device) is not acceptable.  This entry point serves them: it takes plain
// device pointers for the medium, the input and the output, and keeps all of
// its workspace (the per-axis coefficient table, omega^2/c^2 and the three
// Taylor buffers) in one fixed array that is part of the library image.
//
// The array below holds kNoAllocMaxUnknowns unknowns worth of workspace
// (about 16 MB); every GPU that loads the library reserves it until the
// process exits.  Calls share it: two calls whose work overlaps on the GPU
// (different streams, or host threads racing) corrupt each other, so callers
// must order them.  The first call on a device looks up the array's device
// address (cudaGetSymbolAddress).  Every call reads the range of c back to the
// host and synchronises its stream once, because the shift and the Taylor plan
// are chosen on the host from that range (by the same planning code as the
// problem path, plan.cu).
#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>

#include "mxp_internal.h"

namespace {

using cd = std::complex<double>;

constexpr int64_t kNoAllocMaxUnknowns = 1 << 18;    // 262,144 unknowns (e.g. 512 x 512)
constexpr int kNoAllocMaxAxis = 4096;               // unknowns along one axis
constexpr int kNoAllocMaxPml = 64;                  // PML cells per side
// layout in doubles: coefficient table (9 rows of kNoAllocMaxAxis complex),
// omega^2/c^2, three complex buffers, min/max of c
constexpr size_t kCoefOff = 0;
constexpr size_t kKappaOff = kCoefOff + (size_t)9 * kNoAllocMaxAxis * 2;
constexpr size_t kBufOff = kKappaOff + (size_t)kNoAllocMaxUnknowns;
constexpr size_t kMinMaxOff = kBufOff + (size_t)3 * 2 * kNoAllocMaxUnknowns;
constexpr size_t kScratchDoubles = kMinMaxOff + 8;   // min, max, non-finite / non-positive flag

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Error paths only: the message goes to the library's mxp_last_error() slot.
mxp_status nfail(mxp_status s, const char *msg)
{
    mxp::note_error(msg);
    return s;
}

// 1/s at coordinate x for axis d (Eq. pml-1d-s); same formula as the problem setup.
__host__ __device__ inline void inv_stretch_nd(double x, double L, int npml, double h, double cpml,
                                               double omega, double *re, double *im)
{
    if (npml == 0) { *re = 1.0; *im = 0.0; return; }
    const double delta = npml * h;
    double dist = 0.0;
    if (x < 0.0) dist = -x;
    if (x > L) dist = x - L;
    const double r = dist / delta;
    const double b = cpml / (delta * omega) * r * r;   // s = 1 + i b
    const double den = 1.0 + b * b;
    *re = 1.0 / den;
    *im = -b / den;
}

struct AxisGeom {
    int n[3];
    double L[3];
};

__global__ void k_noalloc_coef(AxisGeom ag, int dim, int npml, double h, double cpml, double omega,
                               int nmax)
{
    double2 *coef = reinterpret_cast<double2 *>(g_noalloc_scratch + kCoefOff);
    const double ih2 = 1.0 / (h * h);
    for (int d = 0; d < dim; ++d) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ag.n[d]; i += gridDim.x * blockDim.x) {
            const double x = ((double)i - npml + 0.5) * h;
            double ar, ai, pr, pi, mr, mi;
            inv_stretch_nd(x, ag.L[d], npml, h, cpml, omega, &ar, &ai);
            inv_stretch_nd(x + 0.5 * h, ag.L[d], npml, h, cpml, omega, &pr, &pi);
            inv_stretch_nd(x - 0.5 * h, ag.L[d], npml, h, cpml, omega, &mr, &mi);
            const double2 wp = make_double2((ar * pr - ai * pi) * ih2, (ar * pi + ai * pr) * ih2);
            const double2 wm = make_double2((ar * mr - ai * mi) * ih2, (ar * mi + ai * mr) * ih2);
            coef[(size_t)(3 * d + 0) * nmax + i] = wp;
            coef[(size_t)(3 * d + 1) * nmax + i] = wm;
            coef[(size_t)(3 * d + 2) * nmax + i] = make_double2(wp.x + wm.x, wp.y + wm.y);
        }
    }
}

// kappa = omega^2 / c^2 and min / max of c (one block does the reduction).
__global__ void k_noalloc_kappa(const double *__restrict__ c, double w2, int64_t n)
{
    double *kap = g_noalloc_scratch + kKappaOff;
    __shared__ double smin[256], smax[256];
    double lo = 1e300, hi = 0.0;
    int bad = 0;
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
        const double v = c[p];
        kap[p] = w2 / (v * v);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
        bad |= !(v > 0.0) || !isfinite(v);   // fmin / fmax skip NaN: flag it here
    }
    bad = __syncthreads_or(bad);
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        g_noalloc_scratch[kMinMaxOff] = smin[0];
        g_noalloc_scratch[kMinMaxOff + 1] = smax[0];
        g_noalloc_scratch[kMinMaxOff + 2] = bad ? 1.0 : 0.0;
    }
}

mxp_status scratch_for_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(MXP_ECUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return nfail(MXP_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return MXP_OK;
}

}  // namespace

extern "C" mxp_status mxp_apply_phi_noalloc(const mxp_grid *grid, const mxp_params *prm,
                                            const double *c_dev, int which, const void *x_dev,
                                            void *y_dev, void *cuda_stream, int64_t *passes_out)
{
    using namespace mxp;
    if (!grid || !prm || !c_dev || !x_dev || !y_dev) return nfail(MXP_EINVAL, "NULL argument");
    if (x_dev == y_dev) return nfail(MXP_EINVAL, "x and y must not alias");
    if (which != 0 && which != 1) return nfail(MXP_EINVAL, "which must be 0 (exp) or 1 (psi_1)");
    if (grid->dim != 2 && grid->dim != 3) return nfail(MXP_EINVAL, "dim must be 2 or 3");
    if (grid->npml < 0 || grid->npml > kNoAllocMaxPml)
        return nfail(MXP_EINVAL, "npml must lie in [0, 64] for the allocation-free action");
    if (!(grid->h > 0) || !std::isfinite(grid->h)) return nfail(MXP_EINVAL, "h must be finite and > 0");
    if (!(prm->omega > 0) || !std::isfinite(prm->omega) || !(prm->t > 0) || !std::isfinite(prm->t) ||
        !(prm->c_pml >= 0) || !(prm->shift_s >= 0) || !(prm->exp_tol > 0 && prm->exp_tol < 1) ||
        !(prm->theta_max >= 0 && prm->theta_max <= 30))
        return nfail(MXP_EINVAL, "invalid parameters (omega, t, c_pml, shift_s, exp_tol, theta_max)");
    AxisGeom ag{{1, 1, 1}, {0, 0, 0}};
    int64_t ntot = 1;
    int nmax = 1;
    for (int d = 0; d < grid->dim; ++d) {
        if (grid->n_interior[d] < 1) return nfail(MXP_EINVAL, "n_interior must be >= 1");
        const int64_t nd = grid->n_interior[d] + 2 * (int64_t)grid->npml;
        if (nd > kNoAllocMaxAxis) return nfail(MXP_EINVAL, "an axis exceeds the 4096-unknown limit of the allocation-free action");
        ag.n[d] = (int)nd;
        ag.L[d] = (double)grid->n_interior[d] * grid->h;
        ntot *= nd;
        nmax = std::max(nmax, (int)nd);
    }
    if (ntot > kNoAllocMaxUnknowns)
        return nfail(MXP_EINVAL, "grid exceeds the 262144-unknown limit of the allocation-free action");

    double *scr = nullptr;
    mxp_status s = scratch_for_current_device(&scr);
    if (s != MXP_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double2 *coef = reinterpret_cast<double2 *>(scr + kCoefOff);
    double *kappa = scr + kKappaOff;
    double2 *buf[3] = {reinterpret_cast<double2 *>(scr + kBufOff),
                       reinterpret_cast<double2 *>(scr + kBufOff + 2 * kNoAllocMaxUnknowns),
                       reinterpret_cast<double2 *>(scr + kBufOff + 4 * kNoAllocMaxUnknowns)};

    // per-axis PML coefficients, omega^2/c^2 and the range of c, on the device
    k_noalloc_coef<<<8, 256, 0, st>>>(ag, grid->dim, grid->npml, grid->h, prm->c_pml, prm->omega, nmax);
    k_noalloc_kappa<<<1, 256, 0, st>>>(c_dev, prm->omega * prm->omega, ntot);
    double mm[3] = {0, 0, 0};
    if (cudaMemcpyAsync(mm, scr + kMinMaxOff, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return nfail(MXP_ECUDA, "setting up the allocation-free action failed");
    if (mm[2] != 0.0 || !(mm[0] > 0) || !std::isfinite(mm[1]))
        return nfail(MXP_EINVAL, "wave speed must be finite and > 0");

    // shift mu and Taylor plan from the same host planning code as the problem
    // path: coefficient classes of every PML position plus one interior position
    AxisClasses cls[3];
    const double ih2 = 1.0 / (grid->h * grid->h);
    for (int d = 0; d < grid->dim; ++d) {
        const int n = ag.n[d], p = grid->npml;
        for (int i = 0; i < n; ++i) {
            if (!(i < p || i >= n - p || i == p)) continue;
            const double x = ((double)i - p + 0.5) * grid->h;
            double ar, ai, pr, pi, mr, mi;
            inv_stretch_nd(x, ag.L[d], p, grid->h, prm->c_pml, prm->omega, &ar, &ai);
            inv_stretch_nd(x + 0.5 * grid->h, ag.L[d], p, grid->h, prm->c_pml, prm->omega, &pr, &pi);
            inv_stretch_nd(x - 0.5 * grid->h, ag.L[d], p, grid->h, prm->c_pml, prm->omega, &mr, &mi);
            const cd wp = cd(ar, ai) * cd(pr, pi) * ih2, wm = cd(ar, ai) * cd(mr, mi) * ih2;
            cls[d].off.push_back(std::abs(wp) + std::abs(wm));
            cls[d].wc.push_back(wp + wm);
        }
    }
    const double w2 = prm->omega * prm->omega;
    const ShiftChoice sh = choose_shift(cls, grid->dim, w2 / (mm[1] * mm[1]), w2 / (mm[0] * mm[0]),
                                        prm->shift_s, prm->t);
    const double mu = sh.mu;
    const double nu_plan = which ? std::max(sh.nu, std::abs(prm->t * mu)) : sh.nu;
    const double tol = which ? prm->exp_tol * 0.1 : prm->exp_tol;
    const double theta = prm->theta_max > 0 ? prm->theta_max : 6.0;
    const TaylorPlan plan = make_plan(nu_plan, tol, theta, 1);
    const int Sbest = plan.S, mbest = plan.m;

    // Taylor-Horner sweeps on the shifted (augmented) matrix, as in the problem path
    Geom g{};
    g.dim = grid->dim;
    for (int d = 0; d < 3; ++d) g.n[d] = ag.n[d];
    g.s1 = ag.n[0];
    g.s2 = (int64_t)ag.n[0] * ag.n[1];
    g.ntot = ntot;
    g.nmax = nmax;
    const size_t bytes = (size_t)ntot * sizeof(double2);
    const double2 *v = nullptr;
    if (which == 0) {
        if (cudaMemcpyAsync(buf[0], x_dev, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return nfail(MXP_ECUDA, "copy of the input failed");
    } else {
        if (cudaMemsetAsync(buf[0], 0, bytes, st) != cudaSuccess) return nfail(MXP_ECUDA, "clearing the scratch failed");
        v = static_cast<const double2 *>(x_dev);
    }
    const double t = prm->t;
    const cd rot(0.0, -t * mu / Sbest);
    const cd final_rho = std::exp(cd(0.0, t * mu));
    cd yxi = which ? cd(1.0) : cd(0.0);
    StepScalars<double2> sc;
    sc.zfac = make_double2(1.0, prm->shift_s);
    sc.mu = mu;
    int iy = 0;
    int64_t passes = 0;
    for (int sub = 0; sub < Sbest; ++sub) {
        int in = iy;
        cd pxi = yxi;
        for (int k = mbest; k >= 1; --k) {
            sc.sigma = make_double2(0.0, t / ((double)Sbest * k));
            const cd gam = which ? pxi / ((double)Sbest * k) : cd(0.0);
            sc.gamma = make_double2(gam.real(), gam.imag());
            const cd rho = (sub == Sbest - 1 && k == 1) ? final_rho : cd(1.0);
            sc.rho = make_double2(rho.real(), rho.imag());
            const int o = (in == iy) ? (iy + 1) % 3 : 3 - iy - in;
            launch_step<double2>(g, coef, kappa, sc, buf[in], buf[iy], v, buf[o], st);
            pxi = yxi + rot * pxi / (double)k;
            in = o;
            ++passes;
        }
        iy = in;
        yxi = pxi;
    }
    if (cudaMemcpyAsync(y_dev, buf[iy], bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return nfail(MXP_ECUDA, "copy of the result failed");
    if (cudaGetLastError() != cudaSuccess) return nfail(MXP_ECUDA, "a kernel launch failed");
    if (passes_out) *passes_out = passes;
    return MXP_OK;
}
