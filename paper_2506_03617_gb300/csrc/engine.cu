// Solver engine and C ABI of libmatexpre: problem setup (medium, PML profiles,
// complex shift), the exp / psi_1 actions as shifted Taylor-Horner sweeps,
// Algorithm 1 (inner GMRES on (I - exp(i t A_s)) w = psi_1(i t A_s) r) and the
// outer flexible GMRES (Sec. 3.4).
//
// Matrix functions (Def. psi).  With a real shift mu, M = i t A_s
// = i t mu I + M', M' = i t (A_s - mu I), and exp(M) = e^{i t mu} exp(M').
// psi_1(M) v is the first block of exp(B)[0; 1] for the augmented matrix
// B = [[M, v], [0, 0]]; shifting B by i t mu leaves the scalar row as
// e^{-i t mu tau}, so both actions become exp of a shifted (augmented) matrix
// applied over S sub-steps, each a degree-m Taylor polynomial in Horner form:
//   p <- y + (X p + gamma_k v) / k,  k = m .. 1,  X = M'/S,
// where gamma_k carries the scalar (augmented) component.  mu minimises the
// row-sum norm bound nu = ||t (A_s - mu I)||_inf; (S, m) minimise S*m subject
// to S (nu/S)^(m+1)/(m+1)! e^(nu/S) <= exp_tol and nu/S <= theta_max.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mxp_internal.h"

using namespace mxp;
using cd = std::complex<double>;

static thread_local std::string g_last_error;

void mxp::note_error(const char *msg) { g_last_error = msg; }

static mxp_status fail(mxp_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? MXP_ENOMEM : MXP_ECUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

#define CKS(expr)                                \
    do {                                         \
        mxp_status s_ = (expr);                  \
        if (s_ != MXP_OK) return s_;             \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

struct Arnoldi {
    double2 *V = nullptr;     // (R+1) vectors
    double2 *Z = nullptr;     // R vectors (flexible variant only)
    HessState hs{};
    double2 *tmpcol = nullptr;
    int R = 0;
};

struct mxp_problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    mxp_grid grid{};
    Geom geom{};
    int64_t ntot = 0;
    double cmin = 0, cmax = 0;
    // slab of a larger grid (mxp_create_slab): the problem holds rows
    // [row0, row0 + geom.n[dim-1]) of the last axis of `grid`; coefficients and
    // the Taylor plan follow the global grid, cmin / cmax are the global range
    int slab = 0;
    int64_t row0 = 0;
    mxp_params prm{};
    // device data
    double *c_dev = nullptr;
    double *kappa64 = nullptr;
    float *kappa32 = nullptr;
    double2 *coef64 = nullptr;
    float2 *coef32 = nullptr;
    float2 *coef32s = nullptr;           // coef32 scaled by h^2 in double (persistent kernel)
    // ghost-point faces (mxp_set_boundary): condition per face, and the diagonal
    // term of every boundary cell of a non-Dirichlet face (complex128 and complex64)
    int bc[6] = {0, 0, 0, 0, 0, 0};
    int nfaces = 0;
    double2 *face64 = nullptr;
    float2 *face32 = nullptr;
    float2 *face32s = nullptr;            // face32 scaled by h^2 (persistent kernel)
    int64_t face_off[6] = {0, 0, 0, 0, 0, 0};
    // tensor maps of the TMA-staged 3D sweep (built on first use per precision)
    Tma3Maps *tma3 = nullptr;
    int tma3_prec = -1;                  // precision the maps (or their absence) belong to
    std::vector<double2> coef_host;   // [3][3][nmax]
    // shift and plans
    double mu = 0;
    double nu = 0, nu_aug = 0, nu_aug2 = 0;
    TaylorPlan plan_exp, plan_psi, plan_psi2;
    int fused_cfg = -1;        // tile configuration of the fused 2D sweeps, -1 = unfused
    int fused_tyo = 0;         // output-tile height of the fused sweeps (0 = largest)
    double fused_cost = 1e30;  // estimated ms per exp action with the per-pass kernels
    int persist_cfg = -1;      // persistent exp-action kernel (2D), -1 = not used
    int f3_cfg = -1, f3_lz = 64;   // fused 3D exp sweeps, -1 = unfused
    int p_txo = 0, p_tyo = 0, p_ntx = 0, p_nty = 0;
    float *tau_dev = nullptr;  // per-step tau / h^2 of the exp plan (persistent kernel)
    size_t tau_cap = 0;
    // psi_1 on the persistent kernel: its plan (m a multiple of the kernel's K),
    // per-step tau / h^2 and the sub-step factors c_j = e^{-i t mu j / S}
    TaylorPlan plan_psi_p;
    float *tau_psi_dev = nullptr;
    float2 *wcoef_dev = nullptr;
    size_t tau_psi_cap = 0, wcoef_cap = 0;
    unsigned *bar = nullptr;   // grid-barrier words of the persistent kernel
    // batched solves (several right-hand sides of this problem in lockstep)
    struct Rhs {
        Arnoldi outer, inner;
        double2 *rt = nullptr, *r = nullptr;
    };
    std::vector<Rhs> rhs;
    int bcap = 0;                         // batch slots allocated
    void *bslot[4] = {nullptr, nullptr, nullptr, nullptr};   // bcap vectors each, 16 B per unknown
    double *bhost = nullptr;              // pinned, 8 doubles per right-hand side
    std::map<long long, cudaGraphExec_t> graphs;   // captured pass sequences
    cudaStream_t cap_stream = nullptr;    // private stream the sweep sequences are captured on
    TaylorPlan bplan_exp, bplan_psi;      // plans of the batched (per-pass fused) sweeps
    // workspace
    void *hb[4] = {nullptr, nullptr, nullptr, nullptr};   // 16 bytes per unknown each
    double2 *rt = nullptr, *tmp = nullptr, *tmp2 = nullptr;
    double2 *bdev = nullptr, *xdev = nullptr;
    double2 *vec_dev = nullptr;           // [128]: results of mxp_vec_mdot, coefficients of mxp_vec_combine
    Arnoldi inner, outer;
    KrylovScratch ks{};
    double *host_scal = nullptr;   // pinned, 8 doubles
    // counters
    int64_t passes = 0;
    // learned stage
    mxp_cnn *cnn = nullptr;
    double cnn_tol = 0.5;
};

// ------------------------------------------------------------------ helpers

static cd inv_stretch(const mxp_problem *P, int d, double x)
{
    const int p = P->grid.npml;
    if (p == 0) return 1.0;
    const double h = P->grid.h;
    const double L = (double)P->grid.n_interior[d] * h;
    const double delta = p * h;
    double dist = 0.0;
    if (x < 0.0) dist = -x;
    if (x > L) dist = x - L;
    const double r = dist / delta;
    const cd s(1.0, P->prm.c_pml / (delta * P->prm.omega) * r * r);
    return 1.0 / s;
}

static void build_coef_host(mxp_problem *P)
{
    const int nm = P->geom.nmax;
    const double h = P->grid.h, ih2 = 1.0 / (h * h);
    P->coef_host.assign((size_t)9 * nm, make_double2(0, 0));
    for (int d = 0; d < P->grid.dim; ++d) {
        const int64_t off = (P->slab && d == P->grid.dim - 1) ? P->row0 : 0;   // global index of local row 0
        for (int i = 0; i < P->geom.n[d]; ++i) {
            const double x = ((double)(i + off) - P->grid.npml + 0.5) * h;
            const cd a = inv_stretch(P, d, x);
            const cd bp = inv_stretch(P, d, x + 0.5 * h);
            const cd bm = inv_stretch(P, d, x - 0.5 * h);
            const cd wp = a * bp * ih2, wm = a * bm * ih2, wc = wp + wm;
            P->coef_host[(size_t)(3 * d + 0) * nm + i] = make_double2(wp.real(), wp.imag());
            P->coef_host[(size_t)(3 * d + 1) * nm + i] = make_double2(wm.real(), wm.imag());
            P->coef_host[(size_t)(3 * d + 2) * nm + i] = make_double2(wc.real(), wc.imag());
        }
    }
}

static int effective_fuse(const mxp_problem *P)
{
    return P->fused_cfg >= 0 ? fused2d_cfg_k(P->fused_cfg) : 1;
}

static int exp_fuse(const mxp_problem *P)
{
    if (P->grid.dim == 3) return P->f3_cfg >= 0 ? fused3d_cfg_k(P->f3_cfg) : 1;
    return P->persist_cfg >= 0 ? persist2d_cfg_k(P->persist_cfg) : effective_fuse(P);
}

static double theta_of(const mxp_problem *P)
{
    double theta = P->prm.theta_max;
    if (!(theta > 0)) theta = (P->prm.prec == MXP_C128) ? 6.0 : 4.0;
    return theta;
}

static void make_plans(mxp_problem *P)
{
    P->plan_exp = make_plan(P->nu, P->prm.exp_tol, theta_of(P), exp_fuse(P));
    P->plan_psi = make_plan(P->nu_aug, P->prm.exp_tol * 0.1, theta_of(P), effective_fuse(P));
    P->plan_psi2 = make_plan(P->nu_aug2, P->prm.exp_tol * 0.1, theta_of(P), effective_fuse(P));
    if (P->persist_cfg >= 0)
        P->plan_psi_p = make_plan(P->nu_aug, P->prm.exp_tol * 0.1, theta_of(P), persist2d_cfg_k(P->persist_cfg));
}

// Per-step tau / h^2 of the exp plan for the persistent kernel.
static mxp_status upload_tau(mxp_problem *P)
{
    const TaylorPlan &pl = P->plan_exp;
    const size_t cnt = (size_t)pl.S * pl.m;
    std::vector<float> tau(cnt);
    const double h2 = P->grid.h * P->grid.h;
    for (int sub = 0; sub < pl.S; ++sub)
        for (int k = pl.m; k >= 1; --k)
            tau[(size_t)sub * pl.m + (pl.m - k)] = (float)(P->prm.t / ((double)pl.S * k * h2));
    if (cnt > P->tau_cap) {
        cudaFree(P->tau_dev);
        P->tau_dev = nullptr;
        CK(cudaMalloc(&P->tau_dev, cnt * sizeof(float)));
        P->tau_cap = cnt;
    }
    CK(cudaMemcpyAsync(P->tau_dev, tau.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, P->stream));
    // the psi_1 plan: tau of every step and c_j = e^{-i t mu j / S}, j = 1 .. S-1
    const TaylorPlan &pq = P->plan_psi_p;
    const size_t cq = (size_t)pq.S * pq.m;
    std::vector<float> tq(cq);
    for (int sub = 0; sub < pq.S; ++sub)
        for (int k = pq.m; k >= 1; --k)
            tq[(size_t)sub * pq.m + (pq.m - k)] = (float)(P->prm.t / ((double)pq.S * k * h2));
    std::vector<float2> wc((size_t)std::max(pq.S - 1, 1));
    for (int j = 1; j < pq.S; ++j) {
        const cd c = std::exp(cd(0.0, -P->prm.t * P->mu * j / pq.S));
        wc[(size_t)j - 1] = make_float2((float)c.real(), (float)c.imag());
    }
    if (cq > P->tau_psi_cap) {
        cudaFree(P->tau_psi_dev);
        P->tau_psi_dev = nullptr;
        CK(cudaMalloc(&P->tau_psi_dev, cq * sizeof(float)));
        P->tau_psi_cap = cq;
    }
    if (wc.size() > P->wcoef_cap) {
        cudaFree(P->wcoef_dev);
        P->wcoef_dev = nullptr;
        CK(cudaMalloc(&P->wcoef_dev, wc.size() * sizeof(float2)));
        P->wcoef_cap = wc.size();
    }
    CK(cudaMemcpyAsync(P->tau_psi_dev, tq.data(), cq * sizeof(float), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->wcoef_dev, wc.data(), wc.size() * sizeof(float2), cudaMemcpyHostToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return MXP_OK;
}

static void update_plans(mxp_problem *P)
{
    // per-axis coefficient classes (every PML index plus one interior index of
    // the whole grid, so that every slab of a grid gets the same plan)
    AxisClasses cls[3];
    const double h = P->grid.h, ih2 = 1.0 / (h * h);
    for (int d = 0; d < P->grid.dim; ++d) {
        const int64_t n = P->grid.n_interior[d] + 2 * (int64_t)P->grid.npml, p = P->grid.npml;
        for (int64_t i = 0; i < n; ++i) {
            if (!(i < p || i >= n - p || i == p)) continue;
            const double x = ((double)i - p + 0.5) * h;
            const cd a = inv_stretch(P, d, x), bp = inv_stretch(P, d, x + 0.5 * h), bm = inv_stretch(P, d, x - 0.5 * h);
            const cd wp = a * bp * ih2, wm = a * bm * ih2;
            cls[d].off.push_back(std::abs(wp) + std::abs(wm));
            cls[d].wc.push_back(wp + wm);
        }
    }
    const double w2 = P->prm.omega * P->prm.omega;
    const ShiftChoice sh = choose_shift(cls, P->grid.dim, w2 / (P->cmax * P->cmax), w2 / (P->cmin * P->cmin),
                                        P->prm.shift_s, P->prm.t);
    P->mu = sh.mu;
    P->nu = sh.nu;
    P->nu_aug = std::max(P->nu, std::abs(P->prm.t * P->mu));
    P->nu_aug2 = std::max(P->nu, std::abs(P->prm.t * P->mu) + 1.0);   // Jordan block of psi_2
    make_plans(P);
}

// Float coefficient table for the complex64 / bf16-storage sweeps.  The shift
// mu is folded into the diagonal rows (wc_d + mu/dim, formed in double) so that
// the large, nearly cancelling terms mu and sum_d wc_d never meet in float; the
// float kernels are then called with mu = 0.
static mxp_status upload_coef32(mxp_problem *P)
{
    const size_t cnt = P->coef_host.size();
    const int nm = P->geom.nmax;
    const double h2 = P->grid.h * P->grid.h;
    std::vector<float2> c32(cnt), c32s(cnt);
    for (size_t i = 0; i < cnt; ++i) {
        double re = P->coef_host[i].x;
        const size_t row = i / nm;
        if (row % 3 == 2 && (int)(row / 3) < P->grid.dim) re += P->mu / P->grid.dim;
        c32[i] = make_float2((float)re, (float)P->coef_host[i].y);
        c32s[i] = make_float2((float)(re * h2), (float)(P->coef_host[i].y * h2));
    }
    CK(cudaMemcpyAsync(P->coef32, c32.data(), cnt * sizeof(float2), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->coef32s, c32s.data(), cnt * sizeof(float2), cudaMemcpyHostToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return MXP_OK;
}

static mxp_status upload_coefs(mxp_problem *P)
{
    build_coef_host(P);
    const size_t cnt = P->coef_host.size();
    CK(cudaMemcpyAsync(P->coef64, P->coef_host.data(), cnt * sizeof(double2), cudaMemcpyHostToDevice, P->stream));
    compute_kappa(P->c_dev, P->prm.omega, P->kappa64, P->kappa32, P->ntot, P->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(P->stream));
    return MXP_OK;
}

static mxp_status validate_params(const mxp_params *p)
{
    auto fin = [](double v) { return std::isfinite(v); };
    if (!fin(p->omega) || p->omega <= 0) return fail(MXP_EINVAL, "omega must be finite and > 0");
    if (!fin(p->c_pml) || p->c_pml < 0) return fail(MXP_EINVAL, "c_pml must be finite and >= 0");
    if (!fin(p->shift_s) || p->shift_s < 0) return fail(MXP_EINVAL, "shift_s must be finite and >= 0");
    if (!fin(p->t) || p->t <= 0) return fail(MXP_EINVAL, "t must be finite and > 0");
    if (!fin(p->fprtol) || p->fprtol <= 0 || p->fprtol >= 1) return fail(MXP_EINVAL, "fprtol must lie in (0, 1)");
    if (!fin(p->exp_tol) || p->exp_tol <= 0 || p->exp_tol >= 1) return fail(MXP_EINVAL, "exp_tol must lie in (0, 1)");
    if (p->inner_restart < 1 || p->inner_restart > 64) return fail(MXP_EINVAL, "inner_restart must lie in [1, 64]");
    if (p->inner_maxit < 1) return fail(MXP_EINVAL, "inner_maxit must be >= 1");
    if (p->inner_fixed < 0) return fail(MXP_EINVAL, "inner_fixed must be >= 0");
    if (p->prec != MXP_C128 && p->prec != MXP_C64 && p->prec != MXP_BF16S) return fail(MXP_EINVAL, "unknown precision");
    if (!fin(p->theta_max) || p->theta_max < 0 || p->theta_max > 30) return fail(MXP_EINVAL, "theta_max must lie in [0, 30]");
    if (p->fuse_k < 0 || p->fuse_k > kMaxFuse) return fail(MXP_EINVAL, "fuse_k must lie in [0, 8]");
    if (p->tile_cfg < -1 || p->tile_cfg >= std::max(fused2d_num_cfgs(), fused3d_num_cfgs()))
        return fail(MXP_EINVAL, "tile_cfg out of range");
    if (p->persist_cfg < -2 || p->persist_cfg >= persist2d_num_cfgs()) return fail(MXP_EINVAL, "persist_cfg out of range");
    if (p->precond < 0 || p->precond > 2)
        return fail(MXP_EINVAL, "precond must be 0 (Algorithm 1), 1 (P_N) or 2 (second inverse formula)");
    if (p->neumann_n < 0 || p->neumann_n > 10000) return fail(MXP_EINVAL, "neumann_n must lie in [0, 10000]");
    return MXP_OK;
}

static void free_arnoldi(Arnoldi &a)
{
    cudaFree(a.V); cudaFree(a.Z); cudaFree(a.hs.H); cudaFree(a.hs.cs); cudaFree(a.hs.sn);
    cudaFree(a.hs.g); cudaFree(a.hs.y); cudaFree(a.hs.scal); cudaFree(a.tmpcol);
    a = Arnoldi{};
}

static mxp_status ensure_arnoldi(mxp_problem *P, Arnoldi &a, int R, bool flexible)
{
    if (a.V && a.R >= R && (!flexible || a.Z)) return MXP_OK;
    free_arnoldi(a);
    const int64_t n = P->ntot;
    CK(cudaMalloc(&a.V, (size_t)(R + 1) * n * sizeof(double2)));
    if (flexible) CK(cudaMalloc(&a.Z, (size_t)R * n * sizeof(double2)));
    CK(cudaMalloc(&a.hs.H, (size_t)(R + 1) * R * sizeof(double2)));
    CK(cudaMalloc(&a.hs.cs, R * sizeof(double)));
    CK(cudaMalloc(&a.hs.sn, R * sizeof(double2)));
    CK(cudaMalloc(&a.hs.g, (R + 1) * sizeof(double2)));
    CK(cudaMalloc(&a.hs.y, R * sizeof(double2)));
    CK(cudaMalloc(&a.hs.scal, 8 * sizeof(double)));
    CK(cudaMalloc(&a.tmpcol, (R + 1) * sizeof(double2)));
    CK(cudaMemsetAsync(a.hs.H, 0, (size_t)(R + 1) * R * sizeof(double2), P->stream));
    a.hs.R = R;
    a.R = R;
    return MXP_OK;
}

static mxp_status ensure_base(mxp_problem *P)
{
    const int64_t n = P->ntot;
    for (int i = 0; i < 4; ++i)
        if (!P->hb[i]) CK(cudaMalloc(&P->hb[i], (size_t)n * 16));
    if (!P->rt) CK(cudaMalloc(&P->rt, n * sizeof(double2)));
    if (!P->tmp) CK(cudaMalloc(&P->tmp, n * sizeof(double2)));
    if (!P->tmp2) CK(cudaMalloc(&P->tmp2, n * sizeof(double2)));
    if (!P->ks.partials) {
        P->ks.grid = sm_count() * 4;
        CK(cudaMalloc(&P->ks.partials, (size_t)P->ks.grid * kChunk * sizeof(double2)));
    }
    if (!P->host_scal) CK(cudaMallocHost(&P->host_scal, 8 * sizeof(double)));
    if (!P->bar) {
        // [0..3] grid-barrier words and error flag, [4..] per-tile pass epochs
        CK(cudaMalloc(&P->bar, kPersistBarWords * sizeof(unsigned)));
        CK(cudaMemsetAsync(P->bar, 0, kPersistBarWords * sizeof(unsigned), P->stream));
    }
    return MXP_OK;
}

// Copy `count` device doubles to host_scal[0..count) and the persistent
// kernel's barrier error word alongside; one stream synchronisation.
static mxp_status read_scal(mxp_problem *P, const double *dev, int count)
{
    if (count > 0)
        CK(cudaMemcpyAsync(P->host_scal, dev, count * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    if (P->bar) CK(cudaMemcpyAsync(&P->host_scal[7], P->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (P->bar && *reinterpret_cast<unsigned *>(&P->host_scal[7]) != 0u) {
        CK(cudaMemsetAsync(P->bar, 0, 4 * sizeof(unsigned), P->stream));
        return fail(MXP_ETIMEOUT, "grid barrier of the persistent exp kernel timed out");
    }
    return MXP_OK;
}

// ------------------------------------------------------------------ actions

template <typename S> struct PrecData;
template <> struct PrecData<double2> {
    static const double2 *coef(const mxp_problem *P) { return P->coef64; }
    static const double *kappa(const mxp_problem *P) { return P->kappa64; }
    static const double2 *faces(const mxp_problem *P) { return P->face64; }
    static double2 c(cd z) { return make_double2(z.real(), z.imag()); }
};
template <> struct PrecData<float2> {
    static const float2 *coef(const mxp_problem *P) { return P->coef32; }
    static const float *kappa(const mxp_problem *P) { return P->kappa32; }
    static const float2 *faces(const mxp_problem *P) { return P->face32; }
    static float2 c(cd z) { return make_float2((float)z.real(), (float)z.imag()); }
};

// Point the sweep scalars at the ghost-point face terms of the problem.
template <typename S>
static void set_faces(const mxp_problem *P, StepScalars<typename St<S>::C> &sc)
{
    sc.nfaces = P->nfaces;
    for (int f = 0; f < 6; ++f)
        sc.face[f] = (P->bc[f] != MXP_BC_DIRICHLET) ? PrecData<S>::faces(P) + P->face_off[f] : nullptr;
}
template <> struct PrecData<__nv_bfloat162> : PrecData<float2> {};

template <typename S>
static bool fused_pass(mxp_problem *P, int cfg, const FusedStep *steps, const S *pin, const S *y,
                       const S *v, S *pout)
{
    return launch_fused2d<S>(cfg, P->fused_tyo, P->geom, P->grid.npml, P->coef32, P->kappa32, steps,
                             make_float2(1.0f, (float)P->prm.shift_s), 0.0f,
                             (float)(1.0 / (P->grid.h * P->grid.h)), pin, y, v, pout, P->stream);
}

struct TuneKey {
    int dim, n0, n1, n2, prec, fuse_k;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(dim, n0, n1, n2, prec, fuse_k) < std::tie(o.dim, o.n0, o.n1, o.n2, o.prec, o.fuse_k);
    }
};
static std::map<TuneKey, std::pair<int, int>> g_tuned;
static std::map<TuneKey, double> g_tuned_cost;
static std::map<TuneKey, int> g_tuned_persist;
static std::mutex g_tune_mutex;

// Pick the sweep kernel for a 2D low-precision problem: time a few passes of
// every fused tile configuration (and the unfused kernel) on this grid and
// keep the one with the smallest (sweeps per action) x (time per sweep).
// fuse_k = 1 forces the unfused kernel, fuse_k = K restricts to that K.
// Results are cached per (grid, precision, fuse_k) for the process.
template <typename S>
static mxp_status tune_fused(mxp_problem *P)
{
    P->fused_cfg = -1;
    P->fused_tyo = 0;
    P->fused_cost = 1e30;
    if (P->grid.dim != 2 || P->prm.prec == MXP_C128 || P->prm.fuse_k == 1) return MXP_OK;
    if (P->prm.tile_cfg >= 0) { P->fused_cfg = P->prm.tile_cfg; return MXP_OK; }
    const TuneKey key{P->grid.dim, P->geom.n[0], P->geom.n[1], P->geom.n[2], (int)P->prm.prec, P->prm.fuse_k};
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            P->fused_cfg = it->second.first;
            P->fused_tyo = it->second.second;
            P->fused_cost = g_tuned_cost[key];
            return MXP_OK;
        }
    }
    CKS(ensure_base(P));
    const int64_t n = P->ntot;
    S *b0 = (S *)P->hb[0], *b1 = (S *)P->hb[1], *b2 = (S *)P->hb[2];
    CK(cudaMemsetAsync(b0, 0, (size_t)n * sizeof(S), P->stream));
    CK(cudaMemsetAsync(b1, 0, (size_t)n * sizeof(S), P->stream));
    const int nsm = sm_count();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = -1;
    int best_cfg = -1, best_tyo = 0;
    for (int cfg = -1; cfg < fused2d_num_cfgs(); ++cfg) {
        const int K = cfg >= 0 ? fused2d_cfg_k(cfg) : 1;
        if (P->prm.fuse_k > 1 && K != P->prm.fuse_k) continue;
        // output-tile heights to try: the largest, and heights whose tile count
        // just fits 1..6 waves of two resident CTAs per SM
        std::vector<int> tyos{0};
        if (cfg >= 0) {
            const int maxt = fused2d_cfg_max_tyo(cfg);
            const int txo = fused2d_cfg_rx(cfg) - 2 * K;
            const int ntx = (P->geom.n[0] + txo - 1) / txo;
            for (int waves = 1; waves <= 6; ++waves) {
                const int nty = (waves * 2 * nsm) / ntx;
                if (nty < 1) continue;
                const int tyo = (P->geom.n[1] + nty - 1) / nty;
                if (tyo >= 2 && tyo < maxt &&
                    std::find(tyos.begin(), tyos.end(), tyo) == tyos.end())
                    tyos.push_back(tyo);
            }
        }
        FusedStep steps[kMaxFuse];
        for (int s = 0; s < K; ++s) steps[s] = FusedStep{1e-9, 0, 0, 1, 0, 0};
        const int passes = std::max(4, 96 / K);
        const TaylorPlan pl = make_plan(P->nu, P->prm.exp_tol, theta_of(P), K);
        for (int tyo : tyos) {
            P->fused_tyo = tyo;
            float best_ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, P->stream);
                for (int i = 0; i < passes; ++i) {
                    if (cfg >= 0) {
                        fused_pass<S>(P, cfg, steps, (i & 1) ? b2 : b1, b0, nullptr, (i & 1) ? b1 : b2);
                    } else {
                        StepScalars<typename St<S>::C> sc;
                        sc.zfac = PrecData<S>::c(cd(1.0, P->prm.shift_s));
                        sc.mu = 0;
                        sc.sigma = PrecData<S>::c(cd(0.0, 1e-9));
                        sc.gamma = PrecData<S>::c(cd(0.0));
                        sc.rho = PrecData<S>::c(cd(1.0));
                        launch_step<S>(P->geom, PrecData<S>::coef(P), PrecData<S>::kappa(P), sc,
                                       (i & 1) ? b2 : b1, b0, nullptr, (i & 1) ? b1 : b2, P->stream);
                    }
                }
                cudaEventRecord(e1, P->stream);
                CK(cudaEventSynchronize(e1));
                CK(cudaGetLastError());
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best_ms = std::min(best_ms, ms);   // rep 0 warms up
            }
            const double cost = best_ms / (passes * (double)K) * pl.S * pl.m;
            if (best < 0 || cost < best) { best = cost; best_cfg = cfg; best_tyo = tyo; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->fused_cfg = best_cfg;
    P->fused_tyo = best_tyo;
    P->fused_cost = best;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tuned[key] = {best_cfg, best_tyo};
    g_tuned_cost[key] = best;
    return MXP_OK;
}

// Face terms of a 2D problem for the persistent kernel (h^2-scaled), or nullptr.
struct PersistFaces {
    const float2 *f[4] = {nullptr, nullptr, nullptr, nullptr};
};
static PersistFaces persist_faces(const mxp_problem *P)
{
    PersistFaces pf;
    if (P->nfaces && P->face32s)
        for (int f = 0; f < 4; ++f)
            if (P->bc[f] != MXP_BC_DIRICHLET) pf.f[f] = P->face32s + P->face_off[f];
    return pf;
}

template <typename S>
static cudaError_t persist_action(mxp_problem *P, const S *x, S *out)
{
    const TaylorPlan &pl = P->plan_exp;
    const int K = persist2d_cfg_k(P->persist_cfg);
    const cd rho = std::exp(cd(0.0, P->prm.t * P->mu));
    const PersistFaces pf = persist_faces(P);
    return launch_persist2d<S>(P->persist_cfg, P->geom, P->grid.npml, P->coef32s, P->kappa32,
                               make_float2(1.0f, (float)P->prm.shift_s),
                               (float)(P->grid.h * P->grid.h), P->tau_dev, pl.S * pl.m / K, pl.m / K,
                               make_float2((float)rho.real(), (float)rho.imag()), P->bar, P->p_txo,
                               P->p_tyo, P->p_ntx, P->p_nty, x, (S *)P->hb[2], (S *)P->hb[3], out,
                               P->stream, nullptr, nullptr, P->nfaces ? pf.f : nullptr);
}

// Try the persistent exp-action kernels: time one whole action of each
// configuration that fits the grid and keep it if it beats `best_cost` (ms
// per action of the per-pass kernels).
template <typename S>
static mxp_status tune_persist(mxp_problem *P, double best_cost)
{
    P->persist_cfg = -1;
    if (P->grid.dim != 2 || P->prm.prec == MXP_C128 || P->prm.persist_cfg == -2) return MXP_OK;
    const bool forced = P->prm.persist_cfg >= 0;
    if (!forced && (P->prm.fuse_k == 1 || P->prm.tile_cfg >= 0)) return MXP_OK;
    CKS(ensure_base(P));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = -1, bt[4] = {0, 0, 0, 0};
    for (int id = 0; id < persist2d_num_cfgs(); ++id) {
        if (forced && id != P->prm.persist_cfg) continue;
        if (!forced && P->prm.fuse_k > 1 && persist2d_cfg_k(id) != P->prm.fuse_k) continue;
        if (P->nfaces && !persist2d_cfg_faces(id)) continue;
        int txo, tyo, ntx, nty;
        if (!persist2d_plan<S>(id, P->geom.n[0], P->geom.n[1], P->device, &txo, &tyo, &ntx, &nty)) continue;
        P->persist_cfg = id;
        P->p_txo = txo; P->p_tyo = tyo; P->p_ntx = ntx; P->p_nty = nty;
        make_plans(P);
        CKS(upload_tau(P));
        float best_ms = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaEventRecord(e0, P->stream);
            if (persist_action<S>(P, (const S *)P->hb[0], (S *)P->hb[1]) != cudaSuccess) { ok = false; cudaGetLastError(); break; }
            cudaEventRecord(e1, P->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best_ms = std::min(best_ms, ms);
        }
        CKS(read_scal(P, nullptr, 0));   // barrier error check
        if (ok && (forced || best_ms < best_cost)) {
            best_cost = best_ms;
            best = id;
            bt[0] = txo; bt[1] = tyo; bt[2] = ntx; bt[3] = nty;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->persist_cfg = best;
    P->p_txo = bt[0]; P->p_tyo = bt[1]; P->p_ntx = bt[2]; P->p_nty = bt[3];
    make_plans(P);
    if (best >= 0) CKS(upload_tau(P));
    return MXP_OK;
}

// Pick the 3D exp sweep: time a few passes of each fused z-marching
// configuration (and segment length) and the unfused kernel; keep the one with
// the smallest (sweeps per action) x (time per sweep).  fuse_k as in 2D.
template <typename S>
static mxp_status tune_fused3(mxp_problem *P)
{
    P->f3_cfg = -1;
    if (P->grid.dim != 3 || P->prm.prec == MXP_C128 || P->prm.fuse_k == 1) return MXP_OK;
    if (P->prm.tile_cfg >= 0) {
        if (P->prm.tile_cfg >= fused3d_num_cfgs()) return fail(MXP_EINVAL, "tile_cfg out of range for 3D");
        P->f3_cfg = P->prm.tile_cfg;
        P->f3_lz = 64;
        return MXP_OK;
    }
    CKS(ensure_base(P));
    const int64_t n = P->ntot;
    S *b0 = (S *)P->hb[0], *b1 = (S *)P->hb[1], *b2 = (S *)P->hb[2];
    CK(cudaMemsetAsync(b0, 0, (size_t)n * sizeof(S), P->stream));
    CK(cudaMemsetAsync(b1, 0, (size_t)n * sizeof(S), P->stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = -1;
    int best_cfg = -1, best_lz = 64;
    for (int cfg = -1; cfg < fused3d_num_cfgs(); ++cfg) {
        const int K = cfg >= 0 ? fused3d_cfg_k(cfg) : 1;
        if (P->prm.fuse_k > 1 && K != P->prm.fuse_k) continue;
        const TaylorPlan pl = make_plan(P->nu, P->prm.exp_tol, theta_of(P), K);
        for (int lz : {32, 64, 128}) {
            if (cfg < 0 && lz != 32) continue;
            FusedStep steps[kMaxFuse];
            for (int s = 0; s < K; ++s) steps[s] = FusedStep{1e-9, 0, 0, 1, 0, 0};
            const int passes = std::max(2, 8 / K);
            float best_ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, P->stream);
                for (int i = 0; i < passes; ++i) {
                    if (cfg >= 0) {
                        launch_fused3d<S>(cfg, lz, P->geom, P->coef32, P->kappa32, steps,
                                          make_float2(1.0f, (float)P->prm.shift_s), (i & 1) ? b2 : b1, b0,
                                          (i & 1) ? b1 : b2, P->stream);
                    } else {
                        StepScalars<typename St<S>::C> sc;
                        sc.zfac = PrecData<S>::c(cd(1.0, P->prm.shift_s));
                        sc.mu = 0;
                        sc.sigma = PrecData<S>::c(cd(0.0, 1e-9));
                        sc.gamma = PrecData<S>::c(cd(0.0));
                        sc.rho = PrecData<S>::c(cd(1.0));
                        launch_step<S>(P->geom, PrecData<S>::coef(P), PrecData<S>::kappa(P), sc,
                                       (i & 1) ? b2 : b1, b0, nullptr, (i & 1) ? b1 : b2, P->stream);
                    }
                }
                cudaEventRecord(e1, P->stream);
                CK(cudaEventSynchronize(e1));
                CK(cudaGetLastError());
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best_ms = std::min(best_ms, ms);
            }
            const double cost = best_ms / (passes * (double)K) * pl.S * pl.m;
            if (best < 0 || cost < best) { best = cost; best_cfg = cfg; best_lz = lz; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->f3_cfg = best_cfg;
    P->f3_lz = best_lz;
    return MXP_OK;
}

template <typename S>
static mxp_status retune_t(mxp_problem *P)
{
    CKS(tune_fused<S>(P));
    make_plans(P);
    const TuneKey key{P->grid.dim, P->geom.n[0], P->geom.n[1], P->geom.n[2], (int)P->prm.prec,
                      P->prm.fuse_k * 1000 + P->prm.tile_cfg * 10 + P->prm.persist_cfg};
    int cached = -3;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tuned_persist.find(key);
        if (it != g_tuned_persist.end()) cached = it->second;
    }
    if (cached == -3) {
        CKS(tune_persist<S>(P, P->fused_cost));
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tuned_persist[key] = P->persist_cfg;
    } else if (cached >= 0) {
        int txo, tyo, ntx, nty;
        if (persist2d_plan<S>(cached, P->geom.n[0], P->geom.n[1], P->device, &txo, &tyo, &ntx, &nty)) {
            P->persist_cfg = cached;
            P->p_txo = txo; P->p_tyo = tyo; P->p_ntx = ntx; P->p_nty = nty;
            make_plans(P);
            CKS(upload_tau(P));
        }
    } else {
        P->persist_cfg = -1;
    }
    return MXP_OK;
}

static mxp_status retune(mxp_problem *P)
{
    P->persist_cfg = -1;
    P->f3_cfg = -1;
    if (P->slab) {
        // a slab runs single steps through mxp_horner_step: no tiled kernels
        P->fused_cfg = -1;
        P->fused_cost = 1e30;
        make_plans(P);
        return MXP_OK;
    }
    if (P->nfaces) {
        // the tiled sweeps assume zero ghosts; in 2D the persistent kernel carries
        // the face terms and is used whenever a configuration fits
        P->fused_cfg = -1;
        P->fused_cost = 1e30;
        make_plans(P);
        if (P->grid.dim == 2) {
            if (P->prm.prec == MXP_C64) CKS(tune_persist<float2>(P, P->fused_cost));
            else if (P->prm.prec == MXP_BF16S) CKS(tune_persist<__nv_bfloat162>(P, P->fused_cost));
            make_plans(P);
            if (P->persist_cfg >= 0) CKS(upload_tau(P));
        }
        return MXP_OK;
    }
    if (P->grid.dim == 3) {
        if (P->prm.prec == MXP_C64) CKS(tune_fused3<float2>(P));
        else if (P->prm.prec == MXP_BF16S) CKS(tune_fused3<__nv_bfloat162>(P));
        P->fused_cfg = -1;
        make_plans(P);
        return MXP_OK;
    }
    switch (P->prm.prec) {
    case MXP_C64: CKS(retune_t<float2>(P)); break;
    case MXP_BF16S: CKS(retune_t<__nv_bfloat162>(P)); break;
    default: P->fused_cfg = -1; break;
    }
    make_plans(P);
    if (P->persist_cfg >= 0) CKS(upload_tau(P));
    return MXP_OK;
}

// which = 0: out = exp(i t A_s) x; which = 1: out = psi_1(i t A_s) x.
// out_mode 1 returns x - result instead (the fixed-point operator of Eq. fixed-point).
// Tensor maps for the TMA-staged 3D sweep of this problem, or nullptr when the
// grid or the driver does not allow them (the register-marching sweep is used).
template <typename S>
static const Tma3Maps *tma3_maps(mxp_problem *P)
{
    if (P->grid.dim != 3 || P->nfaces) return nullptr;
    if (P->tma3_prec == (int)P->prm.prec) return P->tma3;
    tma3_destroy(P->tma3);
    P->tma3 = tma3_create<S>(P->geom, P->hb, P->kappa32);
    P->tma3_prec = (int)P->prm.prec;
    return P->tma3;
}

// Scalar part of the augmented matrix of a psi action (which = 1: psi_1, one
// scalar; which = 2: psi_2, a 2x2 Jordan block; which = 0: none), advanced by
// the same truncated Taylor-Horner recursion as the grid block.
struct AugScalars {
    int which;
    cd rot, invS;
    double S;
    cd z1, z2;     // state at the sub-step start
    cd g1, g2;     // Horner values within the sub-step
    AugScalars(int w, cd r, int nsub) : which(w), rot(r), invS(1.0 / nsub), S(nsub)
    {
        z1 = (w == 1) ? cd(1.0) : cd(0.0);
        z2 = (w == 2) ? cd(1.0) : cd(0.0);
        g1 = z1;
        g2 = z2;
    }
    void begin_substep() { g1 = z1; g2 = z2; }
    // coefficient of v in the grid-block update of Horner step k
    cd gamma(int k) const { return which ? g1 / (S * k) : cd(0.0); }
    void step(int k)
    {
        const cd n1 = z1 + (rot * g1 + invS * g2) / (double)k;
        const cd n2 = z2 + rot * g2 / (double)k;
        g1 = n1;
        g2 = n2;
    }
    void end_substep() { z1 = g1; z2 = g2; }
};

template <typename S>
static int64_t phi_action(mxp_problem *P, int which, const double2 *x, double2 *out, int out_mode)
{
    using C = typename St<S>::C;
    const TaylorPlan &pl = which == 2 ? P->plan_psi2 : which ? P->plan_psi : P->plan_exp;
    S *b[3] = {(S *)P->hb[0], (S *)P->hb[1], (S *)P->hb[2]};
    S *vs = (S *)P->hb[3];
    const int64_t n = P->ntot;
    cudaStream_t st = P->stream;
    if (which == 0) {
        launch_convert_in<S>(x, b[0], n, st);
    } else {
        launch_convert_in<S>(x, vs, n, st);
        cudaMemsetAsync(b[0], 0, (size_t)n * sizeof(S), st);
    }
    const double t = P->prm.t;
    const int Ssub = pl.S, m = pl.m;
    const cd rot(0.0, -t * P->mu / Ssub);                 // scalar row of the augmented matrix / S
    const cd final_rho = std::exp(cd(0.0, t * P->mu));    // e^{i t mu}
    // scalar rows of the augmented matrix (Def. psi): psi_1 adds one row whose
    // state xi1 = 1 feeds v into the grid block; psi_2 adds a 2x2 Jordan block,
    // xi1' = xi2, xi2 = 1.  After the shift by -i t mu each scalar also decays
    // as e^{-i t mu tau}.  Per sub-step (time 1/S) the Horner recursion of the
    // scalar part is g <- z + J g / k with J = [[rot, 1/S], [0, rot]], and the
    // grid block takes g1 / (S k) times v.
    AugScalars aug(which, rot, Ssub);
    StepScalars<C> sc;
    sc.zfac = PrecData<S>::c(cd(1.0, P->prm.shift_s));
    sc.mu = (sizeof(S) <= 8) ? (typename St<S>::R)0 : (typename St<S>::R)P->mu;  // float tables carry mu
    set_faces<S>(P, sc);
    int64_t passes = 0;
    int iy = 0;
    if (which == 0 && P->persist_cfg >= 0 && sizeof(S) <= 8) {
        const cudaError_t ce = persist_action<S>(P, b[0], b[1]);
        if (ce != cudaSuccess) {
            fail(MXP_ECUDA, std::string("persistent exp kernel: ") + cudaGetErrorString(ce));
            return -1;
        }
        launch_convert_out<S>(b[1], out, x, out_mode, n, st);
        P->passes += (int64_t)Ssub * m;
        return (int64_t)Ssub * m;
    }
    if (which == 1 && P->persist_cfg >= 0 && sizeof(S) <= 8 && P->plan_psi_p.S > 1 && P->tau_psi_dev) {
        // psi_1 on the persistent kernel.  With u(tau) the solution of u' = M u + v
        // shifted by e^{-i t mu tau}, one sub-step of length 1/S is
        //   u_{j+1} = exp(M'/S) u_j + c_j w,  c_j = e^{-i t mu j / S},
        // where w = u_1 (the first sub-step from u_0 = 0) does not depend on j.
        // The first sub-step runs on the per-point sweep (augmented matrix), the
        // other S - 1 in one persistent launch that adds c_j w after sub-step j.
        const TaylorPlan &pq = P->plan_psi_p;
        const int Kp = persist2d_cfg_k(P->persist_cfg);
        const cd rotq(0.0, -t * P->mu / pq.S);
        AugScalars augq(1, rotq, pq.S);
        augq.begin_substep();
        int in = 0;
        for (int k = pq.m; k >= 1; --k) {
            sc.sigma = PrecData<S>::c(cd(0.0, t / ((double)pq.S * k)));
            sc.gamma = PrecData<S>::c(augq.gamma(k));
            sc.rho = PrecData<S>::c(cd(1.0));
            const int o = (in == 0) ? 1 : 3 - in;           // y = b[0] (zero) throughout
            launch_step<S>(P->geom, PrecData<S>::coef(P), PrecData<S>::kappa(P), sc, b[in], b[0], vs, b[o], st);
            augq.step(k);
            in = o;
        }
        S *w = b[in];                                       // b[1] or b[2]
        S *res = b[3 - in];
        const cudaError_t ce = launch_persist2d<S>(
            P->persist_cfg, P->geom, P->grid.npml, P->coef32s, P->kappa32, make_float2(1.0f, (float)P->prm.shift_s),
            (float)(P->grid.h * P->grid.h), P->tau_psi_dev, (pq.S - 1) * pq.m / Kp, pq.m / Kp,
            make_float2((float)final_rho.real(), (float)final_rho.imag()), P->bar, P->p_txo, P->p_tyo, P->p_ntx,
            P->p_nty, w, b[0], vs, res, st, w, P->wcoef_dev, P->nfaces ? persist_faces(P).f : nullptr);
        if (ce != cudaSuccess) {
            fail(MXP_ECUDA, std::string("persistent psi_1 kernel: ") + cudaGetErrorString(ce));
            return -1;
        }
        launch_convert_out<S>(res, out, x, out_mode, n, st);
        P->passes += (int64_t)pq.S * pq.m;
        return (int64_t)pq.S * pq.m;
    }
    if (which == 0 && P->grid.dim == 3 && P->f3_cfg >= 0 && sizeof(S) <= 8 &&
        m % fused3d_cfg_k(P->f3_cfg) == 0) {
        const int K3 = fused3d_cfg_k(P->f3_cfg);
        for (int sub = 0; sub < Ssub; ++sub) {
            int in = iy;
            for (int k = m; k >= 1; k -= K3) {
                FusedStep steps[kMaxFuse];
                for (int s = 0; s < K3; ++s) {
                    const int kk = k - s;
                    steps[s] = FusedStep{t / ((double)Ssub * kk), 0.0, 0.0, final_rho.real(), final_rho.imag(),
                                         (sub == Ssub - 1 && kk == 1) ? 1 : 0};
                }
                const int o = (in == iy) ? (iy + 1) % 3 : 3 - iy - in;
                launch_fused3d<S>(P->f3_cfg, P->f3_lz, P->geom, P->coef32, P->kappa32, steps,
                                  make_float2(1.0f, (float)P->prm.shift_s), b[in], b[iy], b[o], st);
                in = o;
                passes += K3;
            }
            iy = in;
        }
        launch_convert_out<S>(b[iy], out, x, out_mode, n, st);
        P->passes += passes;
        return passes;
    }
    const int cfg = (sizeof(S) <= 8) ? P->fused_cfg : -1;
    const int K = cfg >= 0 ? fused2d_cfg_k(cfg) : 1;
    if (cfg >= 0 && m % K == 0) {
        for (int sub = 0; sub < Ssub; ++sub) {
            int in = iy;
            aug.begin_substep();
            for (int k = m; k >= 1; k -= K) {
                FusedStep steps[kMaxFuse];
                for (int s = 0; s < K; ++s) {
                    const int kk = k - s;
                    const cd gam = aug.gamma(kk);
                    const bool last = (sub == Ssub - 1 && kk == 1);
                    steps[s] = FusedStep{t / ((double)Ssub * kk), gam.real(), gam.imag(),
                                         final_rho.real(), final_rho.imag(), last ? 1 : 0};
                    aug.step(kk);
                }
                const int o = (in == iy) ? (iy + 1) % 3 : 3 - iy - in;
                fused_pass<S>(P, cfg, steps, b[in], b[iy], which ? vs : nullptr, b[o]);
                in = o;
                passes += K;
            }
            iy = in;
            aug.end_substep();
        }
        launch_convert_out<S>(b[iy], out, x, out_mode, n, st);
        P->passes += passes;
        return passes;
    }
    for (int sub = 0; sub < Ssub; ++sub) {
        int in = iy;
        aug.begin_substep();
        for (int k = m; k >= 1; --k) {
            sc.sigma = PrecData<S>::c(cd(0.0, t / ((double)Ssub * k)));
            sc.gamma = PrecData<S>::c(aug.gamma(k));
            sc.rho = PrecData<S>::c((sub == Ssub - 1 && k == 1) ? final_rho : cd(1.0));
            const int o = (in == iy) ? (iy + 1) % 3 : 3 - iy - in;
            bool done = false;
            if constexpr (sizeof(S) <= 8) {
                // 3D complex64 / bf16: planes staged by TMA (b[i] is work buffer i, v is buffer 3)
                if (const Tma3Maps *tm = tma3_maps<S>(P)) {
                    const cudaError_t ce = launch_step3z_tma<S>(P->geom, PrecData<S>::coef(P), sc, tm, in, iy,
                                                                which ? 3 : -1, b[o], P->bar + 2, st);
                    if (ce != cudaSuccess) {
                        fail(MXP_ECUDA, std::string("TMA 3D sweep: ") + cudaGetErrorString(ce));
                        return -1;
                    }
                    done = true;
                }
            }
            if (!done)
                launch_step<S>(P->geom, PrecData<S>::coef(P), PrecData<S>::kappa(P), sc, b[in], b[iy],
                               which ? vs : nullptr, b[o], st);
            aug.step(k);
            in = o;
            ++passes;
        }
        iy = in;
        aug.end_substep();
    }
    launch_convert_out<S>(b[iy], out, x, out_mode, n, st);
    P->passes += passes;
    return passes;
}

static int64_t phi_dispatch(mxp_problem *P, int which, const double2 *x, double2 *out, int out_mode)
{
    switch (P->prm.prec) {
    case MXP_C64: return phi_action<float2>(P, which, x, out, out_mode);
    case MXP_BF16S: return phi_action<__nv_bfloat162>(P, which, x, out, out_mode);
    default: return phi_action<double2>(P, which, x, out, out_mode);
    }
}

static void apply_op(mxp_problem *P, int shifted, const double2 *x, double2 *y, cudaStream_t st = nullptr)
{
    StepScalars<double2> sc;
    sc.zfac = make_double2(1.0, shifted ? P->prm.shift_s : 0.0);
    sc.mu = 0.0;
    sc.sigma = make_double2(1.0, 0.0);
    sc.gamma = make_double2(0.0, 0.0);
    sc.rho = make_double2(1.0, 0.0);
    set_faces<double2>(P, sc);
    launch_step<double2>(P->geom, P->coef64, P->kappa64, sc, x, nullptr, nullptr, y, st ? st : P->stream);
    P->passes += 1;
}

// One Arnoldi step on V[0..j] -> V[j+1] (the new vector is already in V[j+1]):
// classical Gram-Schmidt, repeated only when the first pass cancelled most of
// w (decided on the device), normalisation and the Givens update.  The first
// multi-dot also takes w itself (it is V[j+1]), which gives ||w||^2 for that
// test without an extra pass.  On GB300 these complex128 passes are bound by
// the FP64 pipe, so each skipped second pass halves their cost.
static void arnoldi_step(mxp_problem *P, Arnoldi &a, int j, cudaStream_t on = nullptr)
{
    const int64_t n = P->ntot;
    cudaStream_t st = on ? on : P->stream;
    double2 *w = a.V + (size_t)(j + 1) * n;
    double2 *col = a.hs.H + (size_t)j * (a.R + 1);
    double *gate = a.hs.scal + 6;
    krylov_mdot(a.V, n, j + 2, w, n, col, 0, P->ks, st);          // col[j+1] = ||w||^2
    krylov_reorth_gate(col, j, gate, st);
    krylov_maxpy(w, a.V, n, j + 1, col, -1.0, n, st);
    krylov_mdot(a.V, n, j + 1, w, n, a.tmpcol, 0, P->ks, st, gate);
    krylov_maxpy(w, a.V, n, j + 1, a.tmpcol, -1.0, n, st, gate);
    krylov_addvec(col, a.tmpcol, j + 1, st, gate);
    krylov_nrm2sq(w, n, a.hs.scal, P->ks, st);
    krylov_scale_invnorm(w, w, a.hs.scal, n, st);
    hess_update(a.hs, j, st);
}

// Algorithm 1.
static mxp_status matexpre_apply(mxp_problem *P, const double2 *r, double2 *w, mxp_apply_stats *stats)
{
    CKS(ensure_base(P));
    const int R = P->prm.inner_restart;
    CKS(ensure_arnoldi(P, P->inner, R, false));
    Arnoldi &a = P->inner;
    const int64_t n = P->ntot;
    cudaStream_t st = P->stream;
    const int64_t passes0 = P->passes;

    // Algorithm 1: r~ = psi_1(i t A_s) r, operator I - exp(i t A_s); on the second
    // inverse formula of Sec. 3.1 (precond = 2): r~ = psi_2 r, operator I - psi_1
    const int rhs_which = P->prm.precond == 2 ? 2 : 1;
    const int op_which = P->prm.precond == 2 ? 1 : 0;
    if (phi_dispatch(P, rhs_which, r, P->rt, 0) < 0) return MXP_ECUDA;
    CK(cudaMemsetAsync(w, 0, n * sizeof(double2), st));
    krylov_nrm2sq(P->rt, n, a.hs.scal, P->ks, st);
    hess_start(a.hs, st);
    krylov_scale_invnorm(a.V, P->rt, a.hs.scal, n, st);
    CK(cudaGetLastError());
    CKS(read_scal(P, a.hs.scal, 4));
    const double zeta = P->host_scal[3];
    if (!std::isfinite(zeta)) return fail(MXP_ENAN, "psi_1(i t A_s) r is not finite");
    int total = 0;
    bool converged = (zeta == 0.0);
    double est = zeta;
    const double tol = P->prm.fprtol * zeta;
    const int fixed = P->prm.inner_fixed;
    const int target = fixed > 0 ? fixed : P->prm.inner_maxit;
    while (!converged && total < target) {
        int j = 0;
        bool stop = false;
        for (; j < R && total < target; ++j) {
            // V[j+1] = (I - exp(i t A_s)) V[j]
            if (phi_dispatch(P, op_which, a.V + (size_t)j * n, a.V + (size_t)(j + 1) * n, 1) < 0)
                return MXP_ECUDA;
            arnoldi_step(P, a, j);
            ++total;
            CK(cudaGetLastError());
            CKS(read_scal(P, a.hs.scal, 3));
            est = P->host_scal[1];
            if (!std::isfinite(est)) return fail(MXP_ENAN, "inner GMRES residual is not finite");
            if (P->host_scal[2] != 0.0) { stop = true; converged = true; ++j; break; }
            if (fixed <= 0 && est <= tol) { stop = true; converged = true; ++j; break; }
        }
        hess_backsolve(a.hs, j, st);
        krylov_maxpy(w, a.V, n, j, a.hs.y, 1.0, n, st);   // w += V y
        if (stop || total >= target) break;
        // restart: residual r~ - (I - exp) w
        if (phi_dispatch(P, op_which, w, P->tmp, 1) < 0) return MXP_ECUDA;
        krylov_sub(P->tmp, P->rt, P->tmp, n, st);
        krylov_nrm2sq(P->tmp, n, a.hs.scal, P->ks, st);
        hess_start(a.hs, st);
        krylov_scale_invnorm(a.V, P->tmp, a.hs.scal, n, st);
        CKS(read_scal(P, a.hs.scal, 4));
        est = P->host_scal[3];
        if (!std::isfinite(est)) return fail(MXP_ENAN, "inner GMRES residual is not finite");
        if (fixed <= 0 && est <= tol) converged = true;
    }
    CK(cudaGetLastError());
    if (stats) {
        stats->inner_iters = total;
        stats->converged = converged ? 1 : 0;
        stats->inner_relres = zeta > 0 ? est / zeta : 0.0;
        stats->stencil_passes = P->passes - passes0;
        stats->pt_updates = stats->stencil_passes * n;
    }
    return MXP_OK;
}

// Truncated Neumann preconditioner P_N of Sec. 3.2 (constant -i t dropped):
// w = (sum_{n=0}^{N} exp(i t A_s)^n) psi_1(i t A_s) r; a fixed linear map.
static mxp_status neumann_apply(mxp_problem *P, const double2 *r, double2 *w, mxp_apply_stats *stats)
{
    CKS(ensure_base(P));
    const int64_t n = P->ntot;
    const int64_t passes0 = P->passes;
    if (phi_dispatch(P, 1, r, w, 0) < 0) return MXP_ECUDA;
    double2 *z = P->rt, *zn = P->tmp;
    krylov_copy(z, w, n, P->stream);
    for (int k = 1; k <= P->prm.neumann_n; ++k) {
        if (phi_dispatch(P, 0, z, zn, 0) < 0) return MXP_ECUDA;
        krylov_add(w, zn, n, P->stream);
        std::swap(z, zn);
    }
    CK(cudaGetLastError());
    CKS(read_scal(P, nullptr, 0));
    if (stats) {
        stats->inner_iters = P->prm.neumann_n;
        stats->converged = 1;
        stats->inner_relres = 0.0;
        stats->stencil_passes = P->passes - passes0;
        stats->pt_updates = stats->stencil_passes * n;
    }
    return MXP_OK;
}

static mxp_status precond_apply(mxp_problem *P, const double2 *r, double2 *w, mxp_apply_stats *stats)
{
    return P->prm.precond == 1 ? neumann_apply(P, r, w, stats) : matexpre_apply(P, r, w, stats);
}

// Outer FGMRES(restart), right-preconditioned by Algorithm 1 (Sec. 3.4).
static mxp_status fgmres_solve(mxp_problem *P, const double2 *b, double2 *x, const mxp_solve_opts *o,
                               mxp_solve_stats *stats)
{
    const auto t0 = std::chrono::steady_clock::now();
    CKS(ensure_base(P));
    const int R = o->restart;
    CKS(ensure_arnoldi(P, P->outer, R, true));
    Arnoldi &a = P->outer;
    const int64_t n = P->ntot;
    cudaStream_t st = P->stream;
    const int64_t passes0 = P->passes;
    double2 *r = P->tmp2;

    krylov_nrm2sq(b, n, a.hs.scal, P->ks, st);
    CKS(read_scal(P, a.hs.scal, 1));
    const double bnorm = std::sqrt(P->host_scal[0]);
    if (!std::isfinite(bnorm)) return fail(MXP_ENAN, "right-hand side is not finite");
    if (!o->x0_given) {
        CK(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
        krylov_copy(r, b, n, st);
    } else {
        apply_op(P, 0, x, r);
        krylov_sub(r, b, r, n, st);
    }
    int total = 0, inner_total = 0, nn_acc = 0, nn_rej = 0;
    bool converged = false;
    double est = 0, relres = 1.0;
    mxp_status status = MXP_OK;
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
        converged = true;
        relres = 0;
    }
    while (!converged) {
        krylov_nrm2sq(r, n, a.hs.scal, P->ks, st);
        hess_start(a.hs, st);
        krylov_scale_invnorm(a.V, r, a.hs.scal, n, st);
        CKS(read_scal(P, a.hs.scal, 4));
        const double beta = P->host_scal[3];
        if (!std::isfinite(beta)) return fail(MXP_ENAN, "outer residual is not finite");
        relres = beta / bnorm;
        if (beta <= o->rtol * bnorm) { converged = true; break; }
        if (total >= o->maxit) { status = MXP_ENOCONV; break; }
        int j = 0;
        for (; j < R && total < o->maxit; ++j) {
            bool nn_used = false;
            if (P->cnn && P->grid.dim == 2) {
                // learned stage: z = net(v_j), kept if min_a ||v_j - a A z|| <= tol (||v_j|| = 1)
                if (cnn_apply_vector(P->cnn, P->geom.n[0], P->geom.n[1], a.V + (size_t)j * n, 1.0,
                                     P->c_dev, P->cmax, a.Z + (size_t)j * n) == MXP_OK) {
                    apply_op(P, 0, a.Z + (size_t)j * n, a.V + (size_t)(j + 1) * n);
                    krylov_mdot(a.V + (size_t)j * n, n, 1, a.V + (size_t)(j + 1) * n, n, a.tmpcol, 0, P->ks, st);
                    krylov_nrm2sq(a.V + (size_t)(j + 1) * n, n, a.hs.scal + 5, P->ks, st);
                    CK(cudaMemcpyAsync(P->host_scal + 1, a.tmpcol, sizeof(double2), cudaMemcpyDeviceToHost, st));
                    CKS(read_scal(P, a.hs.scal + 5, 1));
                    const double az2 = P->host_scal[0];
                    const double dre = P->host_scal[1], dim_ = P->host_scal[2];
                    const double rho2 = az2 > 0 ? 1.0 - (dre * dre + dim_ * dim_) / az2 : 1.0;
                    const double rho = std::sqrt(std::max(0.0, rho2));
                    nn_used = std::isfinite(rho) && rho <= P->cnn_tol;
                    if (nn_used) ++nn_acc; else ++nn_rej;
                }
            }
            if (!nn_used) {
                mxp_apply_stats ast{};
                CKS(precond_apply(P, a.V + (size_t)j * n, a.Z + (size_t)j * n, &ast));
                inner_total += ast.inner_iters;
                apply_op(P, 0, a.Z + (size_t)j * n, a.V + (size_t)(j + 1) * n);
            }
            arnoldi_step(P, a, j);
            ++total;
            CK(cudaGetLastError());
            CKS(read_scal(P, a.hs.scal, 3));
            est = P->host_scal[1];
            if (!std::isfinite(est)) return fail(MXP_ENAN, "outer FGMRES residual is not finite");
            if (P->host_scal[2] != 0.0 || est <= o->rtol * bnorm) { ++j; break; }
        }
        hess_backsolve(a.hs, j, st);
        krylov_maxpy(x, a.Z, n, j, a.hs.y, 1.0, n, st);    // x += Z y
        apply_op(P, 0, x, r);                               // true residual
        krylov_sub(r, b, r, n, st);
        krylov_nrm2sq(r, n, a.hs.scal + 4, P->ks, st);
        CKS(read_scal(P, a.hs.scal + 4, 1));
        relres = std::sqrt(P->host_scal[0]) / bnorm;
        if (!std::isfinite(relres)) return fail(MXP_ENAN, "true residual is not finite");
        if (relres <= o->rtol) { converged = true; break; }
        if (total >= o->maxit) { status = MXP_ENOCONV; break; }
    }
    CK(cudaStreamSynchronize(st));
    if (stats) {
        stats->outer_iters = total;
        stats->inner_iters_total = inner_total;
        stats->converged = converged ? 1 : 0;
        stats->true_relres = relres;
        stats->est_relres = bnorm > 0 ? est / bnorm : 0.0;
        stats->stencil_passes = P->passes - passes0;
        stats->pt_updates = stats->stencil_passes * n;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->nn_accepted = nn_acc;
        stats->nn_rejected = nn_rej;
    }
    if (status == MXP_ENOCONV) return fail(MXP_ENOCONV, "outer FGMRES reached maxit");
    return MXP_OK;
}


// ------------------------------------------------------------------ batched solves
// Several right-hand sides of one problem advance in lockstep: their outer
// FGMRES and inner GMRES iterations run side by side, and every exp / psi_1
// action of the active right-hand sides is one sequence of sweeps over the
// whole batch (one launch per pass covers all vectors).  Each sweep sequence
// is captured once as a CUDA graph per (action, batch size, plan) and replayed.
// Right-hand sides that have converged leave the batch.

static void clear_graphs(mxp_problem *P)
{
    for (auto &kv : P->graphs) cudaGraphExecDestroy(kv.second);
    P->graphs.clear();
}

static void free_batch(mxp_problem *P)
{
    clear_graphs(P);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    P->cap_stream = nullptr;
    for (auto &r : P->rhs) {
        free_arnoldi(r.outer);
        free_arnoldi(r.inner);
        cudaFree(r.rt);
        cudaFree(r.r);
    }
    P->rhs.clear();
    for (int i = 0; i < 4; ++i) { cudaFree(P->bslot[i]); P->bslot[i] = nullptr; }
    if (P->bhost) cudaFreeHost(P->bhost);
    P->bhost = nullptr;
    P->bcap = 0;
}

static mxp_status ensure_batch(mxp_problem *P, int nr, int Rout, int Rin)
{
    const int64_t n = P->ntot;
    if (nr > P->bcap) {
        clear_graphs(P);
        for (int i = 0; i < 4; ++i) { cudaFree(P->bslot[i]); P->bslot[i] = nullptr; }
        if (P->bhost) cudaFreeHost(P->bhost);
        P->bhost = nullptr;
        for (int i = 0; i < 4; ++i) CK(cudaMalloc(&P->bslot[i], (size_t)nr * n * 16));
        CK(cudaMallocHost(&P->bhost, (size_t)nr * 8 * sizeof(double)));
        P->bcap = nr;
    }
    if ((int)P->rhs.size() < nr) P->rhs.resize(nr);
    for (int r = 0; r < nr; ++r) {
        auto &s = P->rhs[r];
        CKS(ensure_arnoldi(P, s.outer, Rout, true));
        CKS(ensure_arnoldi(P, s.inner, Rin, false));
        if (!s.rt) CK(cudaMalloc(&s.rt, n * sizeof(double2)));
        if (!s.r) CK(cudaMalloc(&s.r, n * sizeof(double2)));
    }
    return MXP_OK;
}

// Launch the Horner sweeps of one action over nb batch vectors held in the
// batch slots (input in slot 0, psi_1 source in slot 3).  Returns the slot
// holding the result.
template <typename S>
static int batch_sweeps(mxp_problem *P, int which, int nb, const TaylorPlan &pl, int64_t *passes,
                        cudaStream_t st)
{
    using C = typename St<S>::C;
    const int64_t n = P->ntot;
    S *b[3] = {(S *)P->bslot[0], (S *)P->bslot[1], (S *)P->bslot[2]};
    S *vs = which ? (S *)P->bslot[3] : nullptr;
    const double t = P->prm.t;
    const int Ssub = pl.S, m = pl.m;
    const cd rot(0.0, -t * P->mu / Ssub);
    const cd final_rho = std::exp(cd(0.0, t * P->mu));
    const int cfg = (sizeof(S) <= 8 && P->grid.dim == 2) ? P->fused_cfg : -1;
    const int K = cfg >= 0 ? fused2d_cfg_k(cfg) : 1;
    AugScalars aug(which, rot, Ssub);
    int iy = 0;
    StepScalars<C> sc;
    sc.zfac = PrecData<S>::c(cd(1.0, P->prm.shift_s));
    sc.mu = (sizeof(S) <= 8) ? (typename St<S>::R)0 : (typename St<S>::R)P->mu;
    set_faces<S>(P, sc);
    for (int sub = 0; sub < Ssub; ++sub) {
        int in = iy;
        aug.begin_substep();
        for (int k = m; k >= 1; k -= K) {
            const int o = (in == iy) ? (iy + 1) % 3 : 3 - iy - in;
            if (cfg >= 0) {
                FusedStep steps[kMaxFuse];
                for (int s = 0; s < K; ++s) {
                    const int kk = k - s;
                    const cd gam = aug.gamma(kk);
                    steps[s] = FusedStep{t / ((double)Ssub * kk), gam.real(), gam.imag(), final_rho.real(),
                                         final_rho.imag(), (sub == Ssub - 1 && kk == 1) ? 1 : 0};
                    aug.step(kk);
                }
                launch_fused2d<S>(cfg, P->fused_tyo, P->geom, P->grid.npml, P->coef32, P->kappa32, steps,
                                  make_float2(1.0f, (float)P->prm.shift_s), 0.0f,
                                  (float)(1.0 / (P->grid.h * P->grid.h)), b[in], b[iy], vs, b[o], st, nb);
            } else {
                sc.sigma = PrecData<S>::c(cd(0.0, t / ((double)Ssub * k)));
                sc.gamma = PrecData<S>::c(aug.gamma(k));
                sc.rho = PrecData<S>::c((sub == Ssub - 1 && k == 1) ? final_rho : cd(1.0));
                for (int j = 0; j < nb; ++j)
                    launch_step<S>(P->geom, PrecData<S>::coef(P), PrecData<S>::kappa(P), sc, b[in] + j * n,
                                   b[iy] + j * n, vs ? vs + j * n : nullptr, b[o] + j * n, st);
                aug.step(k);
            }
            in = o;
            *passes += K;
        }
        iy = in;
        aug.end_substep();
    }
    return iy;
}

// out[j] = exp(i t A_s) in[j] (which 0) or psi_1(i t A_s) in[j] (which 1), or
// in[j] - that (out_mode 1), for j < nb; vectors complex128.
template <typename S>
static mxp_status phi_batch_t(mxp_problem *P, int which, int nb, const double2 *const *in,
                              double2 *const *out, int out_mode, int64_t *passes_out)
{
    const int64_t n = P->ntot;
    cudaStream_t st = P->stream;
    const int K = (sizeof(S) <= 8 && P->grid.dim == 2 && P->fused_cfg >= 0) ? fused2d_cfg_k(P->fused_cfg) : 1;
    const TaylorPlan pl = which ? P->plan_psi
                                : make_plan(P->nu, P->prm.exp_tol, theta_of(P), K);
    S *b0 = (S *)P->bslot[0], *vs = (S *)P->bslot[3];
    for (int j = 0; j < nb; ++j) {
        if (which == 0) launch_convert_in<S>(in[j], b0 + j * n, n, st);
        else launch_convert_in<S>(in[j], vs + j * n, n, st);
    }
    if (which == 1) CK(cudaMemsetAsync(b0, 0, (size_t)nb * n * sizeof(S), st));
    const long long key = ((((long long)which * 4096 + nb) * 65536 + pl.S) * 1024 + pl.m) * 64 + K;
    int64_t passes = 0;
    int fin = -1;
    auto it = P->graphs.find(key);
    if (it != P->graphs.end()) CK(cudaGraphLaunch(it->second, st));
    if (it == P->graphs.end()) {
        // first time: record the sweep sequence on the private capture stream
        // (the problem's stream may be the legacy stream, which cannot be
        // captured), instantiate it and launch it on the problem's stream; if
        // capture is unavailable the sweeps run once, directly
        if (!P->cap_stream) CK(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
        const long long l0 = g_launch_count.load();
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool ok = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            fin = batch_sweeps<S>(P, which, nb, pl, &passes, P->cap_stream);
            ok = cudaStreamEndCapture(P->cap_stream, &graph) == cudaSuccess && graph &&
                 cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
        }
        if (ok) {
            P->graphs[key] = exec;
            CK(cudaGraphLaunch(exec, st));
        } else {
            cudaGetLastError();
            g_launch_count.store(l0);
            passes = 0;
            fin = batch_sweeps<S>(P, which, nb, pl, &passes, st);   // nothing ran yet: run once
        }
    } else {
        // the replayed graph holds the sweeps: recompute the result slot, the
        // pass count and the kernel count without launching
        const int cfg = (sizeof(S) <= 8 && P->grid.dim == 2) ? P->fused_cfg : -1;
        const int KK = cfg >= 0 ? fused2d_cfg_k(cfg) : 1;
        int iy = 0;
        for (int sub = 0; sub < pl.S; ++sub) {
            int in2 = iy;
            for (int k = pl.m; k >= 1; k -= KK) {
                in2 = (in2 == iy) ? (iy + 1) % 3 : 3 - iy - in2;
                passes += KK;
            }
            iy = in2;
        }
        fin = iy;
        const int per = (cfg >= 0) ? 1 : nb;
        count_launch((int)((passes / KK) * per));
    }
    S *res = (S *)P->bslot[fin];
    for (int j = 0; j < nb; ++j) launch_convert_out<S>(res + j * n, out[j], in[j], out_mode, n, st);
    CK(cudaGetLastError());
    P->passes += passes * nb;
    if (passes_out) *passes_out = passes;
    return MXP_OK;
}

static mxp_status phi_batch(mxp_problem *P, int which, int nb, const double2 *const *in,
                            double2 *const *out, int out_mode, int64_t *passes)
{
    switch (P->prm.prec) {
    case MXP_C64: return phi_batch_t<float2>(P, which, nb, in, out, out_mode, passes);
    case MXP_BF16S: return phi_batch_t<__nv_bfloat162>(P, which, nb, in, out, out_mode, passes);
    default: return phi_batch_t<double2>(P, which, nb, in, out, out_mode, passes);
    }
}

// Read scal[0..cnt) of every listed right-hand side's Arnoldi state into
// bhost[8*i ...], one synchronisation.
static mxp_status read_batch(mxp_problem *P, const std::vector<int> &ids, bool outer, int first, int cnt)
{
    for (size_t i = 0; i < ids.size(); ++i) {
        const Arnoldi &a = outer ? P->rhs[ids[i]].outer : P->rhs[ids[i]].inner;
        CK(cudaMemcpyAsync(P->bhost + 8 * i, a.hs.scal + first, cnt * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    }
    CK(cudaStreamSynchronize(P->stream));
    return MXP_OK;
}

// Algorithm 1 for the listed right-hand sides in lockstep: out[i] = MatExPre(in[i]).
// The inner GMRES of each one stops at fprtol (or inner_fixed iterations) and,
// in this batched form, after at most inner_restart iterations (no restart).
static mxp_status batch_matexpre(mxp_problem *P, const std::vector<int> &ids, const std::vector<const double2 *> &in,
                                 const std::vector<double2 *> &out, std::vector<int> &inner_iters)
{
    const int nb = (int)ids.size();
    const int64_t n = P->ntot;
    cudaStream_t st = P->stream;
    const int R = P->prm.inner_restart;
    std::vector<double2 *> rts(nb);
    for (int i = 0; i < nb; ++i) rts[i] = P->rhs[ids[i]].rt;
    CKS(phi_batch(P, 1, nb, in.data(), rts.data(), 0, nullptr));
    for (int i = 0; i < nb; ++i) {
        Arnoldi &a = P->rhs[ids[i]].inner;
        CK(cudaMemsetAsync(out[i], 0, n * sizeof(double2), st));
        krylov_nrm2sq(rts[i], n, a.hs.scal, P->ks, st);
        hess_start(a.hs, st);
        krylov_scale_invnorm(a.V, rts[i], a.hs.scal, n, st);
    }
    CKS(read_batch(P, ids, false, 3, 1));
    std::vector<double> zeta(nb);
    std::vector<int> jj(nb, 0);
    std::vector<char> active(nb, 1);
    for (int i = 0; i < nb; ++i) {
        zeta[i] = P->bhost[8 * i];
        if (!std::isfinite(zeta[i])) return fail(MXP_ENAN, "psi_1(i t A_s) r is not finite");
        if (zeta[i] == 0.0) active[i] = 0;
    }
    const int fixed = P->prm.inner_fixed;
    const int jmax = std::min(R, fixed > 0 ? fixed : P->prm.inner_maxit);
    for (int j = 0; j < jmax; ++j) {
        std::vector<int> act;
        std::vector<const double2 *> vin;
        std::vector<double2 *> vout;
        for (int i = 0; i < nb; ++i)
            if (active[i]) {
                Arnoldi &a = P->rhs[ids[i]].inner;
                act.push_back(i);
                vin.push_back(a.V + (size_t)j * n);
                vout.push_back(a.V + (size_t)(j + 1) * n);
            }
        if (act.empty()) break;
        CKS(phi_batch(P, 0, (int)act.size(), vin.data(), vout.data(), 1, nullptr));
        std::vector<int> act_ids;
        for (int i : act) {
            arnoldi_step(P, P->rhs[ids[i]].inner, j);
            act_ids.push_back(ids[i]);
        }
        CK(cudaGetLastError());
        CKS(read_batch(P, act_ids, false, 1, 2));
        for (size_t q = 0; q < act.size(); ++q) {
            const int i = act[q];
            const double est = P->bhost[8 * q], brk = P->bhost[8 * q + 1];
            if (!std::isfinite(est)) return fail(MXP_ENAN, "inner GMRES residual is not finite");
            jj[i] = j + 1;
            if (brk != 0.0 || (fixed <= 0 && est <= P->prm.fprtol * zeta[i])) active[i] = 0;
        }
    }
    for (int i = 0; i < nb; ++i) {
        inner_iters[i] = jj[i];
        if (jj[i] == 0) continue;
        Arnoldi &a = P->rhs[ids[i]].inner;
        hess_backsolve(a.hs, jj[i], st);
        krylov_maxpy(out[i], a.V, n, jj[i], a.hs.y, 1.0, n, st);
    }
    CK(cudaGetLastError());
    return MXP_OK;
}

// Outer FGMRES for nr right-hand sides of one problem in lockstep.
static mxp_status batch_solve(mxp_problem *P, int nr, const double2 *const *b, double2 *const *x,
                              const mxp_solve_opts *o, mxp_solve_stats *stats)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (P->prm.precond != 0) return fail(MXP_EINVAL, "batched solves use Algorithm 1 (precond = 0)");
    CKS(ensure_base(P));
    const int R = o->restart;
    CKS(ensure_batch(P, nr, R, P->prm.inner_restart));
    const int64_t n = P->ntot;
    cudaStream_t st = P->stream;
    const int64_t passes0 = P->passes;
    std::vector<int> all(nr);
    for (int r = 0; r < nr; ++r) all[r] = r;
    for (int r = 0; r < nr; ++r) krylov_nrm2sq(b[r], n, P->rhs[r].outer.hs.scal, P->ks, st);
    CKS(read_batch(P, all, true, 0, 1));
    std::vector<double> bnorm(nr), relres(nr, 1.0), est(nr, 0.0);
    std::vector<int> total(nr, 0), inner_total(nr, 0), jr(nr, 0);
    std::vector<char> done(nr, 0), conv(nr, 0);
    for (int r = 0; r < nr; ++r) {
        bnorm[r] = std::sqrt(P->bhost[8 * r]);
        if (!std::isfinite(bnorm[r])) return fail(MXP_ENAN, "right-hand side is not finite");
        if (!o->x0_given) {
            CK(cudaMemsetAsync(x[r], 0, n * sizeof(double2), st));
            krylov_copy(P->rhs[r].r, b[r], n, st);
        } else {
            apply_op(P, 0, x[r], P->rhs[r].r);
            krylov_sub(P->rhs[r].r, b[r], P->rhs[r].r, n, st);
        }
        if (bnorm[r] == 0.0) {
            CK(cudaMemsetAsync(x[r], 0, n * sizeof(double2), st));
            done[r] = conv[r] = 1;
            relres[r] = 0;
        }
    }
    while (true) {
        std::vector<int> live;
        for (int r = 0; r < nr; ++r)
            if (!done[r]) live.push_back(r);
        if (live.empty()) break;
        // cycle start: V0 = r / beta
        for (int r : live) {
            Arnoldi &a = P->rhs[r].outer;
            krylov_nrm2sq(P->rhs[r].r, n, a.hs.scal, P->ks, st);
            hess_start(a.hs, st);
            krylov_scale_invnorm(a.V, P->rhs[r].r, a.hs.scal, n, st);
        }
        CKS(read_batch(P, live, true, 3, 1));
        std::vector<int> cyc;
        for (size_t q = 0; q < live.size(); ++q) {
            const int r = live[q];
            const double beta = P->bhost[8 * q];
            if (!std::isfinite(beta)) return fail(MXP_ENAN, "outer residual is not finite");
            relres[r] = beta / bnorm[r];
            jr[r] = 0;
            if (beta <= o->rtol * bnorm[r]) { done[r] = conv[r] = 1; continue; }
            if (total[r] >= o->maxit) { done[r] = 1; continue; }
            cyc.push_back(r);
        }
        if (cyc.empty()) continue;
        std::vector<char> stop(nr, 0);
        for (int j = 0; j < R; ++j) {
            std::vector<int> act;
            for (int r : cyc)
                if (!stop[r] && total[r] < o->maxit) act.push_back(r);
            if (act.empty()) break;
            std::vector<const double2 *> vin;
            std::vector<double2 *> zout;
            for (int r : act) {
                vin.push_back(P->rhs[r].outer.V + (size_t)j * n);
                zout.push_back(P->rhs[r].outer.Z + (size_t)j * n);
            }
            std::vector<int> inn(act.size(), 0);
            CKS(batch_matexpre(P, act, vin, zout, inn));
            for (size_t q = 0; q < act.size(); ++q) {
                const int r = act[q];
                inner_total[r] += inn[q];
                Arnoldi &a = P->rhs[r].outer;
                apply_op(P, 0, a.Z + (size_t)j * n, a.V + (size_t)(j + 1) * n);
                arnoldi_step(P, a, j);
            }
            CK(cudaGetLastError());
            CKS(read_batch(P, act, true, 1, 2));
            for (size_t q = 0; q < act.size(); ++q) {
                const int r = act[q];
                est[r] = P->bhost[8 * q];
                if (!std::isfinite(est[r])) return fail(MXP_ENAN, "outer FGMRES residual is not finite");
                ++total[r];
                jr[r] = j + 1;
                if (P->bhost[8 * q + 1] != 0.0 || est[r] <= o->rtol * bnorm[r]) stop[r] = 1;
            }
        }
        for (int r : cyc) {
            Arnoldi &a = P->rhs[r].outer;
            hess_backsolve(a.hs, jr[r], st);
            krylov_maxpy(x[r], a.Z, n, jr[r], a.hs.y, 1.0, n, st);
            apply_op(P, 0, x[r], P->rhs[r].r);
            krylov_sub(P->rhs[r].r, b[r], P->rhs[r].r, n, st);
            krylov_nrm2sq(P->rhs[r].r, n, a.hs.scal + 4, P->ks, st);
        }
        CKS(read_batch(P, cyc, true, 4, 1));
        for (size_t q = 0; q < cyc.size(); ++q) {
            const int r = cyc[q];
            relres[r] = std::sqrt(P->bhost[8 * q]) / bnorm[r];
            if (!std::isfinite(relres[r])) return fail(MXP_ENAN, "true residual is not finite");
            if (relres[r] <= o->rtol) done[r] = conv[r] = 1;
            else if (total[r] >= o->maxit) done[r] = 1;
        }
    }
    CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all_conv = true;
    for (int r = 0; r < nr; ++r) {
        all_conv = all_conv && conv[r];
        if (stats) {
            stats[r].outer_iters = total[r];
            stats[r].inner_iters_total = inner_total[r];
            stats[r].converged = conv[r];
            stats[r].true_relres = relres[r];
            stats[r].est_relres = bnorm[r] > 0 ? est[r] / bnorm[r] : 0.0;
            stats[r].stencil_passes = (P->passes - passes0) / std::max(nr, 1);
            stats[r].pt_updates = (P->passes - passes0) * n / std::max(nr, 1);
            stats[r].seconds = secs;
        }
    }
    if (!all_conv) return fail(MXP_ENOCONV, "outer FGMRES reached maxit for a right-hand side");
    return MXP_OK;
}

// ------------------------------------------------------------------ grouped solves
// Sources of several 2D problems (different grids and media, one precision)
// advance in lockstep as one group.  Every pass of an exp / psi_1 action is ONE
// launch of the grouped fused kernel over all (problem, source, tile) items; a
// device mask switches converged sources off, so the pass sequence of each
// action type is captured once as a CUDA graph and replayed for every subset of
// live sources.  The Krylov work (FP64) stays per source on the group's stream.
// All problems share one Taylor plan, made for the largest norm bound of the
// group (extra terms only add accuracy); each problem keeps its own t, shift,
// PML and psi_1 scalars.

struct GroupSource {
    mxp_problem *P;
    int local;     // the source's batch slot in its problem
};

template <typename S>
static mxp_status group_solve_t(const std::vector<mxp_problem *> &probs, const std::vector<std::vector<int>> &rhs_of,
                                const void *const *b_dev, void *const *x_dev, const mxp_solve_opts *o,
                                std::vector<mxp_solve_stats> &out_stats)
{
    const auto t0 = std::chrono::steady_clock::now();
    const int np = (int)probs.size();
    mxp_problem *P0 = probs[0];
    cudaStream_t st = P0->stream;
    for (auto *P : probs) CK(cudaStreamSynchronize(P->stream));
    std::vector<GroupSource> src;
    std::vector<int> caller, src0(np);
    for (int p = 0; p < np; ++p) {
        src0[p] = (int)src.size();
        for (size_t q = 0; q < rhs_of[p].size(); ++q) {
            src.push_back({probs[p], (int)q});
            caller.push_back(rhs_of[p][q]);
        }
    }
    const int ns = (int)src.size();
    const int R = o->restart;
    for (int p = 0; p < np; ++p) {
        CKS(ensure_base(probs[p]));
        CKS(ensure_batch(probs[p], (int)rhs_of[p].size(), R, probs[p]->prm.inner_restart));
    }
    // tile configuration: the largest problem's tuned fused configuration
    int big = 0;
    for (int p = 1; p < np; ++p)
        if (probs[p]->ntot > probs[big]->ntot) big = p;
    int cfg = probs[big]->fused_cfg;
    for (int p = 0; p < np && cfg < 0; ++p) cfg = probs[p]->fused_cfg;
    if (cfg < 0) cfg = 1;
    const int K = fused2d_cfg_k(cfg);
    double nu = 0, nua = 0, tol = 1.0, theta = 1e30;
    for (auto *P : probs) {
        nu = std::max(nu, P->nu);
        nua = std::max(nua, P->nu_aug);
        tol = std::min(tol, P->prm.exp_tol);
        theta = std::min(theta, theta_of(P));
    }
    const TaylorPlan plan[2] = {make_plan(nu, tol, theta, K), make_plan(nua, tol * 0.1, theta, K)};
    // work items and per-problem tables
    std::vector<GroupProblem> gp(np);
    std::vector<int4> bmap;
    for (int p = 0; p < np; ++p) {
        mxp_problem *P = probs[p];
        GroupProblem &g = gp[p];
        g.n0 = P->geom.n[0];
        g.n1 = P->geom.n[1];
        g.npml = P->grid.npml;
        g.nmax = P->geom.nmax;
        int ntx = 0, nty = 0;
        fused2d_tiles(cfg, g.n0, g.n1, P->fused_cfg == cfg ? P->fused_tyo : 0, &g.txo, &g.tyo, &ntx, &nty);
        g.coef = P->coef32;
        g.kappa = P->kappa32;
        for (int i = 0; i < 4; ++i) g.slot[i] = P->bslot[i];
        g.src0 = src0[p];
        for (int j = 0; j < (int)rhs_of[p].size(); ++j)
            for (int by = 0; by < nty; ++by)
                for (int bx = 0; bx < ntx; ++bx) bmap.push_back(make_int4(p, j, bx, by));
    }
    // pass sequences (slot rotation shared by all problems) and their scalars
    struct Pass { int in, iy, o; };
    std::vector<Pass> seq[2];
    std::vector<FusedScalars> sct[2];
    int fin[2] = {0, 0};
    for (int w = 0; w < 2; ++w) {
        const TaylorPlan &pl = plan[w];
        std::vector<AugScalars> aug;
        for (auto *P : probs) aug.emplace_back(w, cd(0.0, -P->prm.t * P->mu / pl.S), pl.S);
        int iy = 0;
        for (int sub = 0; sub < pl.S; ++sub) {
            int in = iy;
            for (auto &a : aug) a.begin_substep();
            for (int k = pl.m; k >= 1; k -= K) {
                const int ob = (in == iy) ? (iy + 1) % 3 : 3 - iy - in;
                seq[w].push_back({in, iy, ob});
                for (int p = 0; p < np; ++p) {
                    mxp_problem *P = probs[p];
                    const cd rho = std::exp(cd(0.0, P->prm.t * P->mu));
                    FusedStep steps[kMaxFuse];
                    for (int q = 0; q < K; ++q) {
                        const int kk = k - q;
                        const cd gam = aug[p].gamma(kk);
                        steps[q] = FusedStep{P->prm.t / ((double)pl.S * kk), gam.real(), gam.imag(), rho.real(),
                                             rho.imag(), (sub == pl.S - 1 && kk == 1) ? 1 : 0};
                        aug[p].step(kk);
                    }
                    FusedScalars fs;
                    fused2d_scalars(cfg, steps, make_float2(1.0f, (float)P->prm.shift_s), 0.0f,
                                    (float)(1.0 / (P->grid.h * P->grid.h)), &fs);
                    sct[w].push_back(fs);
                }
                in = ob;
            }
            iy = in;
            for (auto &a : aug) a.end_substep();
        }
        fin[w] = iy;
    }
    // device copies (freed at the end of the call)
    GroupProblem *gp_dev = nullptr;
    int4 *bmap_dev = nullptr;
    FusedScalars *sc_dev[2] = {nullptr, nullptr};
    int *active_dev = nullptr;
    double *hbuf = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    struct Cleanup {
        std::vector<void *> dev;
        double *host = nullptr;
        cudaGraphExec_t *g = nullptr;
        ~Cleanup()
        {
            for (void *d : dev) cudaFree(d);
            if (host) cudaFreeHost(host);
            for (int w = 0; w < 2; ++w)
                if (g[w]) cudaGraphExecDestroy(g[w]);
        }
    } cleanup;
    cleanup.g = graph;
    CK(cudaMalloc(&gp_dev, np * sizeof(GroupProblem)));
    cleanup.dev.push_back(gp_dev);
    CK(cudaMalloc(&bmap_dev, bmap.size() * sizeof(int4)));
    cleanup.dev.push_back(bmap_dev);
    for (int w = 0; w < 2; ++w) {
        CK(cudaMalloc(&sc_dev[w], sct[w].size() * sizeof(FusedScalars)));
        cleanup.dev.push_back(sc_dev[w]);
        CK(cudaMemcpyAsync(sc_dev[w], sct[w].data(), sct[w].size() * sizeof(FusedScalars), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMalloc(&active_dev, ns * sizeof(int)));
    cleanup.dev.push_back(active_dev);
    CK(cudaMallocHost(&hbuf, (size_t)ns * 8 * sizeof(double)));
    cleanup.host = hbuf;
    CK(cudaMemcpyAsync(gp_dev, gp.data(), np * sizeof(GroupProblem), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(bmap_dev, bmap.data(), bmap.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    const int nblocks = (int)bmap.size();
    auto launch_passes = [&](int w, cudaStream_t on) {
        for (size_t q = 0; q < seq[w].size(); ++q)
            launch_fused2d_group<S>(cfg, gp_dev, bmap_dev, nblocks, sc_dev[w] + q * np, active_dev, seq[w][q].in,
                                    seq[w][q].iy, w ? 3 : -1, seq[w][q].o, on);
    };
    // capture each action type's pass sequence once (private stream; the caller's
    // stream may be the legacy stream); without capture the passes run directly
    if (!P0->cap_stream) CK(cudaStreamCreateWithFlags(&P0->cap_stream, cudaStreamNonBlocking));
    for (int w = 0; w < 2; ++w) {
        const long long l0 = g_launch_count.load();
        cudaGraph_t gr = nullptr;
        bool ok = cudaStreamBeginCapture(P0->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            launch_passes(w, P0->cap_stream);
            ok = cudaStreamEndCapture(P0->cap_stream, &gr) == cudaSuccess && gr &&
                 cudaGraphInstantiate(&graph[w], gr, 0) == cudaSuccess;
            if (gr) cudaGraphDestroy(gr);
        }
        if (!ok) {
            cudaGetLastError();
            graph[w] = nullptr;
        }
        g_launch_count.store(l0);
    }
    std::vector<int> active_h(ns, 0);
    std::vector<int64_t> passes_src(ns, 0);
    // out[q] = action w of in[q] (or in[q] minus it, out_mode 1) for the listed sources
    auto phi_group = [&](int w, const std::vector<int> &ids, const std::vector<const double2 *> &in,
                         const std::vector<double2 *> &out, int out_mode) -> mxp_status {
        for (size_t q = 0; q < ids.size(); ++q) {
            const GroupSource &g = src[ids[q]];
            const int64_t n = g.P->ntot;
            launch_convert_in<S>(in[q], (S *)g.P->bslot[w ? 3 : 0] + g.local * n, n, st);
            if (w) CK(cudaMemsetAsync((S *)g.P->bslot[0] + g.local * n, 0, (size_t)n * sizeof(S), st));
        }
        std::fill(active_h.begin(), active_h.end(), 0);
        for (int id : ids) active_h[id] = 1;
        // pageable source: the copy is staged before the call returns
        CK(cudaMemcpyAsync(active_dev, active_h.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
        if (graph[w]) {
            CK(cudaGraphLaunch(graph[w], st));
            count_launch((int)seq[w].size());
        } else {
            launch_passes(w, st);
        }
        for (size_t q = 0; q < ids.size(); ++q) {
            const GroupSource &g = src[ids[q]];
            const int64_t n = g.P->ntot;
            launch_convert_out<S>((S *)g.P->bslot[fin[w]] + g.local * n, out[q], in[q], out_mode, n, st);
            passes_src[ids[q]] += (int64_t)plan[w].S * plan[w].m;
            g.P->passes += (int64_t)plan[w].S * plan[w].m;
        }
        CK(cudaGetLastError());
        return MXP_OK;
    };
    auto rhs_of_src = [&](int id) -> mxp_problem::Rhs & { return src[id].P->rhs[src[id].local]; };
    auto nof = [&](int id) { return src[id].P->ntot; };
    auto read_group = [&](const std::vector<int> &ids, bool outer, int first, int cnt) -> mxp_status {
        for (size_t q = 0; q < ids.size(); ++q) {
            const Arnoldi &a = outer ? rhs_of_src(ids[q]).outer : rhs_of_src(ids[q]).inner;
            CK(cudaMemcpyAsync(hbuf + 8 * q, a.hs.scal + first, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
        return MXP_OK;
    };
    // Algorithm 1 for the listed sources in lockstep (inner GMRES capped at the
    // restart length, as in the single-problem batched form)
    auto matexpre_group = [&](const std::vector<int> &ids, const std::vector<const double2 *> &in,
                              const std::vector<double2 *> &out, std::vector<int> &inner_iters) -> mxp_status {
        const int nb = (int)ids.size();
        std::vector<double2 *> rts(nb);
        for (int i = 0; i < nb; ++i) rts[i] = rhs_of_src(ids[i]).rt;
        CKS(phi_group(1, ids, in, rts, 0));
        for (int i = 0; i < nb; ++i) {
            mxp_problem *P = src[ids[i]].P;
            Arnoldi &a = rhs_of_src(ids[i]).inner;
            CK(cudaMemsetAsync(out[i], 0, nof(ids[i]) * sizeof(double2), st));
            krylov_nrm2sq(rts[i], nof(ids[i]), a.hs.scal, P->ks, st);
            hess_start(a.hs, st);
            krylov_scale_invnorm(a.V, rts[i], a.hs.scal, nof(ids[i]), st);
        }
        CKS(read_group(ids, false, 3, 1));
        std::vector<double> zeta(nb);
        std::vector<int> jj(nb, 0);
        std::vector<char> act(nb, 1);
        for (int i = 0; i < nb; ++i) {
            zeta[i] = hbuf[8 * i];
            if (!std::isfinite(zeta[i])) return fail(MXP_ENAN, "psi_1(i t A_s) r is not finite");
            if (zeta[i] == 0.0) act[i] = 0;
        }
        int jcap = 0;
        for (int i = 0; i < nb; ++i) jcap = std::max(jcap, src[ids[i]].P->prm.inner_restart);
        for (int j = 0; j < jcap; ++j) {
            std::vector<int> live, live_ids;
            std::vector<const double2 *> vin;
            std::vector<double2 *> vout;
            for (int i = 0; i < nb; ++i) {
                const mxp_problem *P = src[ids[i]].P;
                const int fixed = P->prm.inner_fixed;
                const int jmax = std::min(P->prm.inner_restart, fixed > 0 ? fixed : P->prm.inner_maxit);
                if (!act[i] || j >= jmax) continue;
                Arnoldi &a = rhs_of_src(ids[i]).inner;
                live.push_back(i);
                live_ids.push_back(ids[i]);
                vin.push_back(a.V + (size_t)j * nof(ids[i]));
                vout.push_back(a.V + (size_t)(j + 1) * nof(ids[i]));
            }
            if (live.empty()) break;
            CKS(phi_group(0, live_ids, vin, vout, 1));
            for (int i : live) arnoldi_step(src[ids[i]].P, rhs_of_src(ids[i]).inner, j, st);
            CK(cudaGetLastError());
            CKS(read_group(live_ids, false, 1, 2));
            for (size_t q = 0; q < live.size(); ++q) {
                const int i = live[q];
                const mxp_problem *P = src[ids[i]].P;
                const double est = hbuf[8 * q], brk = hbuf[8 * q + 1];
                if (!std::isfinite(est)) return fail(MXP_ENAN, "inner GMRES residual is not finite");
                jj[i] = j + 1;
                if (brk != 0.0 || (P->prm.inner_fixed <= 0 && est <= P->prm.fprtol * zeta[i])) act[i] = 0;
            }
        }
        for (int i = 0; i < nb; ++i) {
            inner_iters[i] = jj[i];
            if (jj[i] == 0) continue;
            Arnoldi &a = rhs_of_src(ids[i]).inner;
            hess_backsolve(a.hs, jj[i], st);
            krylov_maxpy(out[i], a.V, nof(ids[i]), jj[i], a.hs.y, 1.0, nof(ids[i]), st);
        }
        CK(cudaGetLastError());
        return MXP_OK;
    };

    // outer FGMRES of every source in lockstep
    std::vector<const double2 *> b(ns);
    std::vector<double2 *> x(ns);
    for (int r = 0; r < ns; ++r) {
        b[r] = (const double2 *)b_dev[caller[r]];
        x[r] = (double2 *)x_dev[caller[r]];
    }
    std::vector<int> all(ns);
    for (int r = 0; r < ns; ++r) all[r] = r;
    for (int r = 0; r < ns; ++r) krylov_nrm2sq(b[r], nof(r), rhs_of_src(r).outer.hs.scal, src[r].P->ks, st);
    CKS(read_group(all, true, 0, 1));
    std::vector<double> bnorm(ns), relres(ns, 1.0), est(ns, 0.0), secs(ns, 0.0);
    std::vector<int> total(ns, 0), inner_total(ns, 0), jr(ns, 0);
    std::vector<char> done(ns, 0), conv(ns, 0);
    auto now = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    for (int r = 0; r < ns; ++r) {
        bnorm[r] = std::sqrt(hbuf[8 * r]);
        if (!std::isfinite(bnorm[r])) return fail(MXP_ENAN, "right-hand side is not finite");
        if (!o->x0_given) {
            CK(cudaMemsetAsync(x[r], 0, nof(r) * sizeof(double2), st));
            krylov_copy(rhs_of_src(r).r, b[r], nof(r), st);
        } else {
            apply_op(src[r].P, 0, x[r], rhs_of_src(r).r, st);
            krylov_sub(rhs_of_src(r).r, b[r], rhs_of_src(r).r, nof(r), st);
        }
        if (bnorm[r] == 0.0) {
            CK(cudaMemsetAsync(x[r], 0, nof(r) * sizeof(double2), st));
            done[r] = conv[r] = 1;
            relres[r] = 0;
        }
    }
    while (true) {
        std::vector<int> live;
        for (int r = 0; r < ns; ++r)
            if (!done[r]) live.push_back(r);
        if (live.empty()) break;
        for (int r : live) {
            Arnoldi &a = rhs_of_src(r).outer;
            krylov_nrm2sq(rhs_of_src(r).r, nof(r), a.hs.scal, src[r].P->ks, st);
            hess_start(a.hs, st);
            krylov_scale_invnorm(a.V, rhs_of_src(r).r, a.hs.scal, nof(r), st);
        }
        CKS(read_group(live, true, 3, 1));
        std::vector<int> cyc;
        for (size_t q = 0; q < live.size(); ++q) {
            const int r = live[q];
            const double beta = hbuf[8 * q];
            if (!std::isfinite(beta)) return fail(MXP_ENAN, "outer residual is not finite");
            relres[r] = beta / bnorm[r];
            jr[r] = 0;
            if (beta <= o->rtol * bnorm[r]) { done[r] = conv[r] = 1; secs[r] = now(); continue; }
            if (total[r] >= o->maxit) { done[r] = 1; secs[r] = now(); continue; }
            cyc.push_back(r);
        }
        if (cyc.empty()) continue;
        std::vector<char> stop(ns, 0);
        for (int j = 0; j < R; ++j) {
            std::vector<int> act;
            for (int r : cyc)
                if (!stop[r] && total[r] < o->maxit) act.push_back(r);
            if (act.empty()) break;
            std::vector<const double2 *> vin;
            std::vector<double2 *> zout;
            for (int r : act) {
                vin.push_back(rhs_of_src(r).outer.V + (size_t)j * nof(r));
                zout.push_back(rhs_of_src(r).outer.Z + (size_t)j * nof(r));
            }
            std::vector<int> inn(act.size(), 0);
            CKS(matexpre_group(act, vin, zout, inn));
            for (size_t q = 0; q < act.size(); ++q) {
                const int r = act[q];
                inner_total[r] += inn[q];
                Arnoldi &a = rhs_of_src(r).outer;
                apply_op(src[r].P, 0, a.Z + (size_t)j * nof(r), a.V + (size_t)(j + 1) * nof(r), st);
                passes_src[r] += 1;
                arnoldi_step(src[r].P, a, j, st);
            }
            CK(cudaGetLastError());
            CKS(read_group(act, true, 1, 2));
            for (size_t q = 0; q < act.size(); ++q) {
                const int r = act[q];
                est[r] = hbuf[8 * q];
                if (!std::isfinite(est[r])) return fail(MXP_ENAN, "outer FGMRES residual is not finite");
                ++total[r];
                jr[r] = j + 1;
                if (hbuf[8 * q + 1] != 0.0 || est[r] <= o->rtol * bnorm[r]) stop[r] = 1;
            }
        }
        for (int r : cyc) {
            Arnoldi &a = rhs_of_src(r).outer;
            hess_backsolve(a.hs, jr[r], st);
            krylov_maxpy(x[r], a.Z, nof(r), jr[r], a.hs.y, 1.0, nof(r), st);
            apply_op(src[r].P, 0, x[r], rhs_of_src(r).r, st);
            passes_src[r] += 1;
            krylov_sub(rhs_of_src(r).r, b[r], rhs_of_src(r).r, nof(r), st);
            krylov_nrm2sq(rhs_of_src(r).r, nof(r), a.hs.scal + 4, src[r].P->ks, st);
        }
        CKS(read_group(cyc, true, 4, 1));
        for (size_t q = 0; q < cyc.size(); ++q) {
            const int r = cyc[q];
            relres[r] = std::sqrt(hbuf[8 * q]) / bnorm[r];
            if (!std::isfinite(relres[r])) return fail(MXP_ENAN, "true residual is not finite");
            if (relres[r] <= o->rtol) { done[r] = conv[r] = 1; secs[r] = now(); }
            else if (total[r] >= o->maxit) { done[r] = 1; secs[r] = now(); }
        }
    }
    CK(cudaStreamSynchronize(st));
    bool all_conv = true;
    for (int r = 0; r < ns; ++r) {
        all_conv = all_conv && conv[r];
        mxp_solve_stats &sr = out_stats[caller[r]];
        sr.outer_iters = total[r];
        sr.inner_iters_total = inner_total[r];
        sr.converged = conv[r];
        sr.true_relres = relres[r];
        sr.est_relres = bnorm[r] > 0 ? est[r] / bnorm[r] : 0.0;
        sr.stencil_passes = passes_src[r];
        sr.pt_updates = passes_src[r] * nof(r);
        sr.seconds = secs[r];
    }
    if (!all_conv) return fail(MXP_ENOCONV, "outer FGMRES reached maxit for a right-hand side");
    return MXP_OK;
}

// Whether a problem can join a grouped solve (2D, complex64 or bf16 storage,
// zero Dirichlet faces, Algorithm 1).
static bool groupable(const mxp_problem *P)
{
    return P->grid.dim == 2 && (P->prm.prec == MXP_C64 || P->prm.prec == MXP_BF16S) && P->nfaces == 0 &&
           P->prm.precond == 0;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *mxp_status_string(mxp_status s)
{
    switch (s) {
    case MXP_OK: return "ok";
    case MXP_EINVAL: return "invalid argument";
    case MXP_ENOMEM: return "out of memory";
    case MXP_ECUDA: return "CUDA error";
    case MXP_ENOCONV: return "not converged";
    case MXP_EBREAKDOWN: return "Krylov breakdown";
    case MXP_ENAN: return "NaN or Inf";
    case MXP_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *mxp_last_error(void) { return g_last_error.c_str(); }

int64_t mxp_kernel_launch_count(void) { return (int64_t)g_launch_count.load(); }

mxp_status mxp_default_params(const mxp_grid *grid, double c_min, double ppw, mxp_params *p)
{
    if (!grid || !p) return fail(MXP_EINVAL, "NULL argument");
    if (!(grid->h > 0) || !(c_min > 0) || !(ppw > 0)) return fail(MXP_EINVAL, "h, c_min and ppw must be > 0");
    const double h = grid->h;
    const double freq = 1.0 / (ppw * h);
    std::memset(p, 0, sizeof(*p));
    p->omega = 2.0 * M_PI * c_min / (ppw * h);
    p->c_pml = 20.0;
    p->shift_s = 1.0 / freq;
    p->t = 40.0 * h * h;
    p->fprtol = 0.08;
    p->exp_tol = 1e-12;
    p->inner_restart = 30;
    p->inner_maxit = 1000;
    p->inner_fixed = 0;
    p->prec = MXP_C128;
    p->theta_max = 0.0;
    p->fuse_k = 0;
    p->tile_cfg = -1;
    p->persist_cfg = -1;
    p->precond = 0;
    p->neumann_n = 4;
    return MXP_OK;
}

// A problem on rows [row0, row0 + nrows) of the last axis of `grid` (the whole
// grid when nrows < 0).  c_host covers those rows; crange (nullable) gives the
// wave-speed range of the whole grid, which sets the shift and the Taylor plan.
static mxp_status create_impl(const mxp_grid *grid, int64_t row0, int64_t nrows, const double *c_host,
                              const double *crange, int device, void *cuda_stream, mxp_problem **out)
{
    if (!grid || !c_host || !out) return fail(MXP_EINVAL, "NULL argument");
    *out = nullptr;
    if (grid->dim != 2 && grid->dim != 3) return fail(MXP_EINVAL, "dim must be 2 or 3");
    if (grid->npml < 0) return fail(MXP_EINVAL, "npml must be >= 0");
    if (!(grid->h > 0) || !std::isfinite(grid->h)) return fail(MXP_EINVAL, "h must be finite and > 0");
    int64_t ntot = 1;
    int n[3] = {1, 1, 1};
    for (int d = 0; d < grid->dim; ++d) {
        if (grid->n_interior[d] < 1) return fail(MXP_EINVAL, "n_interior must be >= 1");
        const int64_t nd = grid->n_interior[d] + 2 * (int64_t)grid->npml;
        if (nd > (1 << 20)) return fail(MXP_EINVAL, "axis too long");
        n[d] = (int)nd;
    }
    const bool slab = nrows >= 0;
    if (slab) {
        const int last = grid->dim - 1;
        if (row0 < 0 || nrows < 1 || row0 + nrows > n[last])
            return fail(MXP_EINVAL, "slab rows must lie inside the last axis of the grid");
        n[last] = (int)nrows;
    }
    for (int d = 0; d < grid->dim; ++d) ntot *= n[d];
    if (ntot > (int64_t)1 << 34) return fail(MXP_EINVAL, "grid too large");
    double cmin = 1e300, cmax = 0;
    for (int64_t i = 0; i < ntot; ++i) {
        const double v = c_host[i];
        if (!std::isfinite(v) || v <= 0) return fail(MXP_EINVAL, "wave speed must be finite and > 0 everywhere");
        cmin = std::min(cmin, v);
        cmax = std::max(cmax, v);
    }
    if (crange) {
        if (!(crange[0] > 0) || !(crange[1] >= crange[0]) || !std::isfinite(crange[1]) || crange[0] > cmin ||
            crange[1] < cmax)
            return fail(MXP_EINVAL, "the global wave-speed range must be finite, positive and contain the slab's");
        cmin = crange[0];
        cmax = crange[1];
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(MXP_EINVAL, "no such CUDA device");
    DeviceGuard guard(device);
    mxp_problem *P = new mxp_problem();
    P->device = device;
    P->stream = (cudaStream_t)cuda_stream;
    P->grid = *grid;
    P->slab = slab ? 1 : 0;
    P->row0 = slab ? row0 : 0;
    P->geom.dim = grid->dim;
    for (int d = 0; d < 3; ++d) P->geom.n[d] = n[d];
    P->geom.s1 = n[0];
    P->geom.s2 = (int64_t)n[0] * n[1];
    P->geom.ntot = ntot;
    P->geom.nmax = std::max(n[0], std::max(n[1], n[2]));
    // the interior fast path of k_step tests local indices against npml: off for slabs
    P->geom.fast = slab ? 0 : 1;
    P->geom.npml = grid->npml;
    P->geom.ih2 = 1.0 / (grid->h * grid->h);
    P->ntot = ntot;
    P->cmin = cmin;
    P->cmax = cmax;
    mxp_default_params(grid, cmin, 10.0, &P->prm);
    auto bail = [&](mxp_status s) { mxp_destroy(P); return s; };
    const size_t cnt = (size_t)9 * P->geom.nmax;
    if (cudaMalloc(&P->c_dev, ntot * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->kappa64, ntot * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->kappa32, ntot * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&P->coef64, cnt * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&P->coef32, cnt * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&P->coef32s, cnt * sizeof(float2)) != cudaSuccess)
        return bail(fail(MXP_ENOMEM, "device allocation failed"));
    if (cudaMemcpyAsync(P->c_dev, c_host, ntot * sizeof(double), cudaMemcpyHostToDevice, P->stream) != cudaSuccess)
        return bail(fail(MXP_ECUDA, "copy of the medium failed"));
    mxp_status s = upload_coefs(P);
    if (s != MXP_OK) return bail(s);
    update_plans(P);
    s = upload_coef32(P);
    if (s == MXP_OK) s = retune(P);
    if (s != MXP_OK) return bail(s);
    *out = P;
    return MXP_OK;
}

mxp_status mxp_create(const mxp_grid *grid, const double *c_host, int device, void *cuda_stream,
                      mxp_problem **out)
{
    return create_impl(grid, 0, -1, c_host, nullptr, device, cuda_stream, out);
}

mxp_status mxp_create_slab(const mxp_grid *grid, int64_t row0, int64_t nrows, const double *c_slab_host,
                           const double *c_range, int device, void *cuda_stream, mxp_problem **out)
{
    if (!c_range) return fail(MXP_EINVAL, "NULL argument");
    return create_impl(grid, row0, nrows, c_slab_host, c_range, device, cuda_stream, out);
}

mxp_status mxp_horner_step(mxp_problem *P, const double *sigma, const double *gamma, const double *rho,
                           const void *p_dev, const void *y_dev, const void *v_dev, void *out_dev)
{
    if (!P || !sigma || !rho || !p_dev || !out_dev || (v_dev && !gamma)) return fail(MXP_EINVAL, "NULL argument");
    if (out_dev == p_dev || out_dev == y_dev || out_dev == v_dev)
        return fail(MXP_EINVAL, "out must not alias p, y or v");
    DeviceGuard guard(P->device);
    StepScalars<double2> sc;
    sc.zfac = make_double2(1.0, P->prm.shift_s);
    sc.mu = P->mu;
    sc.sigma = make_double2(sigma[0], sigma[1]);
    sc.gamma = v_dev ? make_double2(gamma[0], gamma[1]) : make_double2(0.0, 0.0);
    sc.rho = make_double2(rho[0], rho[1]);
    set_faces<double2>(P, sc);
    launch_step<double2>(P->geom, P->coef64, P->kappa64, sc, (const double2 *)p_dev, (const double2 *)y_dev,
                         (const double2 *)v_dev, (double2 *)out_dev, P->stream);
    P->passes += 1;
    CK(cudaGetLastError());
    return MXP_OK;
}

static mxp_status ensure_vec(mxp_problem *P)
{
    if (!P->ks.partials) {
        P->ks.grid = sm_count() * 4;
        CK(cudaMalloc(&P->ks.partials, (size_t)P->ks.grid * kChunk * sizeof(double2)));
    }
    if (!P->vec_dev) CK(cudaMalloc(&P->vec_dev, 128 * sizeof(double2)));
    return MXP_OK;
}

mxp_status mxp_vec_mdot(mxp_problem *P, const void *V_dev, int64_t ldv, int k, const void *w_dev, int64_t row_lo,
                        int64_t row_hi, double *out_host)
{
    if (!P || !V_dev || !w_dev || !out_host) return fail(MXP_EINVAL, "NULL argument");
    const int64_t nrow = P->geom.n[P->grid.dim - 1], row_len = P->ntot / nrow;
    if (k < 1 || k > 64) return fail(MXP_EINVAL, "k must lie in [1, 64]");
    if (k > 1 && ldv < P->ntot) return fail(MXP_EINVAL, "ldv must be at least the number of unknowns");
    if (row_lo < 0 || row_hi > nrow || row_lo > row_hi) return fail(MXP_EINVAL, "rows outside the problem");
    DeviceGuard guard(P->device);
    CKS(ensure_vec(P));
    if (row_hi == row_lo) {
        for (int i = 0; i < 2 * k; ++i) out_host[i] = 0.0;
        return MXP_OK;
    }
    const int64_t off = row_lo * row_len, len = (row_hi - row_lo) * row_len;
    krylov_mdot((const double2 *)V_dev + off, ldv, k, (const double2 *)w_dev + off, len, P->vec_dev, 0, P->ks,
                P->stream);
    CK(cudaMemcpyAsync(out_host, P->vec_dev, (size_t)k * sizeof(double2), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return MXP_OK;
}

mxp_status mxp_vec_combine(mxp_problem *P, void *y_dev, const double *beta, const void *V_dev, int64_t ldv, int k,
                           const double *coef_host)
{
    if (!P || !y_dev || !beta || (k > 0 && (!V_dev || !coef_host))) return fail(MXP_EINVAL, "NULL argument");
    if (k < 0 || k > 64) return fail(MXP_EINVAL, "k must lie in [0, 64]");
    if (k > 1 && ldv < P->ntot) return fail(MXP_EINVAL, "ldv must be at least the number of unknowns");
    DeviceGuard guard(P->device);
    CKS(ensure_vec(P));
    const int64_t n = P->ntot;
    if (beta[0] == 0.0 && beta[1] == 0.0)
        CK(cudaMemsetAsync(y_dev, 0, (size_t)n * sizeof(double2), P->stream));   // y is not read
    else if (!(beta[0] == 1.0 && beta[1] == 0.0))
        krylov_scale((double2 *)y_dev, make_double2(beta[0], beta[1]), n, P->stream);
    if (k > 0) {
        CK(cudaMemcpyAsync(P->vec_dev + 64, coef_host, (size_t)k * sizeof(double2), cudaMemcpyHostToDevice, P->stream));
        krylov_maxpy((double2 *)y_dev, (const double2 *)V_dev, ldv, k, P->vec_dev + 64, 1.0, n, P->stream);
    }
    CK(cudaGetLastError());
    return MXP_OK;
}

mxp_status mxp_get_plan(const mxp_problem *P, int which, double *mu, int *S, int *m)
{
    if (!P || !mu || !S || !m) return fail(MXP_EINVAL, "NULL argument");
    if (which < 0 || which > 2) return fail(MXP_EINVAL, "which must be 0 (exp), 1 (psi_1) or 2 (psi_2)");
    const TaylorPlan &pl = which == 2 ? P->plan_psi2 : which ? P->plan_psi : P->plan_exp;
    *mu = P->mu;
    *S = pl.S;
    *m = pl.m;
    return MXP_OK;
}

// Diagonal terms of the ghost-point faces.  A face row's missing neighbour
// coefficient w (a b-/h^2 at index 0, a b+/h^2 at index n_d - 1) multiplies the
// ghost value f u_p: f = 1 on a sound-hard face; on a first-order absorbing face
// (du/dn = i k u, k = omega / c_p, centred difference and mean at the face)
// f = (1 + i k h/2) / (1 - i k h/2).
static mxp_status build_faces(mxp_problem *P)
{
    const int dim = P->grid.dim, nm = P->geom.nmax;
    const int n[3] = {P->geom.n[0], P->geom.n[1], P->geom.n[2]};
    int64_t total = 0;
    for (int f = 0; f < 2 * dim; ++f) {
        P->face_off[f] = total;
        if (P->bc[f] != MXP_BC_DIRICHLET) total += P->ntot / n[f / 2];
    }
    cudaFree(P->face64);
    cudaFree(P->face32);
    cudaFree(P->face32s);
    P->face64 = nullptr;
    P->face32 = nullptr;
    P->face32s = nullptr;
    if (total == 0) return MXP_OK;
    std::vector<double> c((size_t)P->ntot);
    CK(cudaMemcpy(c.data(), P->c_dev, (size_t)P->ntot * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double2> f64((size_t)total);
    std::vector<float2> f32((size_t)total), f32s((size_t)total);
    const double h2 = P->grid.h * P->grid.h;
    const double h = P->grid.h, omega = P->prm.omega;
    for (int f = 0; f < 2 * dim; ++f) {
        if (P->bc[f] == MXP_BC_DIRICHLET) continue;
        const int d = f / 2, side = f % 2;
        const int e = side ? n[d] - 1 : 0;                       // index along the face normal
        const double2 wv = P->coef_host[(size_t)(3 * d + (side ? 0 : 1)) * nm + e];
        const cd w(wv.x, wv.y);
        // the face's cells in the order the sweep indexes them: the two other
        // axes, the lower one fastest
        const int a0 = (d == 0) ? 1 : 0, a1 = (d == 2) ? 1 : 2;
        const int m0 = n[a0], m1 = (dim == 3) ? n[a1] : 1;
        for (int u1 = 0; u1 < m1; ++u1)
            for (int u0 = 0; u0 < m0; ++u0) {
                int idx[3] = {0, 0, 0};
                idx[d] = e;
                idx[a0] = u0;
                if (dim == 3) idx[a1] = u1;
                const int64_t q = idx[0] + (int64_t)n[0] * (idx[1] + (int64_t)n[1] * idx[2]);
                cd gf(1.0);
                if (P->bc[f] == MXP_BC_ABSORBING) {
                    const double kh2 = 0.5 * omega / c[(size_t)q] * h;
                    gf = cd(1.0, kh2) / cd(1.0, -kh2);
                }
                const cd term = w * gf;
                const size_t o = (size_t)(P->face_off[f] + u0 + (int64_t)m0 * u1);
                f64[o] = make_double2(term.real(), term.imag());
                f32[o] = make_float2((float)term.real(), (float)term.imag());
                f32s[o] = make_float2((float)(term.real() * h2), (float)(term.imag() * h2));
            }
    }
    CK(cudaMalloc(&P->face64, (size_t)total * sizeof(double2)));
    CK(cudaMalloc(&P->face32, (size_t)total * sizeof(float2)));
    CK(cudaMalloc(&P->face32s, (size_t)total * sizeof(float2)));
    CK(cudaMemcpyAsync(P->face64, f64.data(), (size_t)total * sizeof(double2), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->face32, f32.data(), (size_t)total * sizeof(float2), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->face32s, f32s.data(), (size_t)total * sizeof(float2), cudaMemcpyHostToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return MXP_OK;
}

mxp_status mxp_set_boundary(mxp_problem *P, const int *bc)
{
    if (!P || !bc) return fail(MXP_EINVAL, "NULL argument");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    for (int f = 0; f < 6; ++f) {
        if (bc[f] < MXP_BC_DIRICHLET || bc[f] > MXP_BC_ABSORBING) return fail(MXP_EINVAL, "unknown boundary condition");
        if (f >= 2 * P->grid.dim && bc[f] != MXP_BC_DIRICHLET)
            return fail(MXP_EINVAL, "faces beyond the grid's dimension must be MXP_BC_DIRICHLET");
    }
    DeviceGuard guard(P->device);
    int nf = 0;
    for (int f = 0; f < 6; ++f) {
        P->bc[f] = bc[f];
        nf += (bc[f] != MXP_BC_DIRICHLET);
    }
    P->nfaces = nf;
    CKS(build_faces(P));
    clear_graphs(P);
    return retune(P);
}

int mxp_sweep_kernel(mxp_problem *P)
{
    if (!P) return -1;
    if (P->persist_cfg >= 0) return MXP_SWEEP_PERSISTENT_2D;
    if (P->grid.dim == 2) return P->fused_cfg >= 0 ? MXP_SWEEP_FUSED_2D : MXP_SWEEP_POINTWISE;
    if (P->f3_cfg >= 0) return MXP_SWEEP_FUSED_3D;
    if (P->prm.prec == MXP_C128) return MXP_SWEEP_POINTWISE;
    if (P->nfaces) return MXP_SWEEP_POINTWISE;
    DeviceGuard guard(P->device);
    if (ensure_base(P) != MXP_OK) return -1;
    const Tma3Maps *tm = (P->prm.prec == MXP_C64) ? tma3_maps<float2>(P) : tma3_maps<__nv_bfloat162>(P);
    return tm ? MXP_SWEEP_ZMARCH_TMA_3D : MXP_SWEEP_ZMARCH_3D;
}

mxp_status mxp_get_boundary(const mxp_problem *P, int *bc)
{
    if (!P || !bc) return fail(MXP_EINVAL, "NULL argument");
    for (int f = 0; f < 6; ++f) bc[f] = P->bc[f];
    return MXP_OK;
}

mxp_status mxp_set_params(mxp_problem *P, const mxp_params *p)
{
    if (!P) return fail(MXP_EINVAL, "NULL problem");
    mxp_params np;
    if (p) np = *p;
    else mxp_default_params(&P->grid, P->cmin, 10.0, &np);
    CKS(validate_params(&np));
    DeviceGuard guard(P->device);
    const bool recoef = np.omega != P->prm.omega || np.c_pml != P->prm.c_pml;
    P->prm = np;
    if (recoef) CKS(upload_coefs(P));
    if (recoef && P->nfaces) CKS(build_faces(P));
    update_plans(P);
    CKS(upload_coef32(P));
    clear_graphs(P);
    return retune(P);
}

mxp_status mxp_get_params(const mxp_problem *P, mxp_params *p)
{
    if (!P || !p) return fail(MXP_EINVAL, "NULL argument");
    *p = P->prm;
    return MXP_OK;
}

int64_t mxp_num_unknowns(const mxp_problem *P) { return P ? P->ntot : 0; }

int mxp_num_tile_configs(void) { return fused2d_num_cfgs(); }

int mxp_num_persist_configs(void) { return persist2d_num_cfgs(); }

mxp_status mxp_selftest_barrier_timeout(mxp_problem *P)
{
    if (!P) return fail(MXP_EINVAL, "NULL problem");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    DeviceGuard guard(P->device);
    CKS(ensure_base(P));
    CK(barrier_selftest(P->bar, P->stream));
    // a persistent launch between the timed-out wait and the host's read must not
    // erase the error word (it finds the word set and leaves its pass loop)
    if (P->persist_cfg >= 0) {
        const cudaError_t ce = (P->prm.prec == MXP_BF16S)
                                   ? persist_action<__nv_bfloat162>(P, (const __nv_bfloat162 *)P->hb[0],
                                                                    (__nv_bfloat162 *)P->hb[1])
                                   : persist_action<float2>(P, (const float2 *)P->hb[0], (float2 *)P->hb[1]);
        CK(ce);
    }
    return read_scal(P, nullptr, 0);   // MXP_ETIMEOUT when the wait ran out (and clears it)
}

mxp_status mxp_attach_cnn(mxp_problem *P, mxp_cnn *net, double accept_tol)
{
    if (!P) return fail(MXP_EINVAL, "NULL problem");
    if (net && !(accept_tol >= 0 && accept_tol <= 1)) return fail(MXP_EINVAL, "accept_tol must lie in [0, 1]");
    if (net && P->grid.dim != 2) return fail(MXP_EINVAL, "the learned stage is available for 2D problems");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    P->cnn = net;
    P->cnn_tol = accept_tol;
    return MXP_OK;
}

int mxp_persist_config(const mxp_problem *P, int *ntiles)
{
    if (!P) return -1;
    if (ntiles) *ntiles = P->persist_cfg >= 0 ? P->p_ntx * P->p_nty : 0;
    return P->persist_cfg;
}

int mxp_persist_geometry(const mxp_problem *P, int *txo, int *tyo, int *ntx, int *nty, int *k)
{
    if (!P || !txo || !tyo || !ntx || !nty || !k) return -1;
    *txo = P->p_txo;
    *tyo = P->p_tyo;
    *ntx = P->p_ntx;
    *nty = P->p_nty;
    *k = P->persist_cfg >= 0 ? persist2d_cfg_k(P->persist_cfg) : 0;
    return P->persist_cfg;
}

int mxp_tile_config(const mxp_problem *P, int *fuse_k)
{
    if (!P) return -1;
    if (P->grid.dim == 3) {
        if (fuse_k) *fuse_k = P->f3_cfg >= 0 ? fused3d_cfg_k(P->f3_cfg) : 1;
        return P->f3_cfg;
    }
    if (fuse_k) *fuse_k = effective_fuse(P);
    return P->fused_cfg;
}

mxp_status mxp_apply_operator(mxp_problem *P, int shifted, const void *x_dev, void *y_dev)
{
    if (!P || !x_dev || !y_dev) return fail(MXP_EINVAL, "NULL argument");
    if (x_dev == y_dev) return fail(MXP_EINVAL, "x and y must not alias");
    DeviceGuard guard(P->device);
    apply_op(P, shifted ? 1 : 0, (const double2 *)x_dev, (double2 *)y_dev);
    CK(cudaGetLastError());
    return MXP_OK;
}

mxp_status mxp_apply_phi(mxp_problem *P, int which, const void *x_dev, void *y_dev, int64_t *passes_out)
{
    if (!P || !x_dev || !y_dev) return fail(MXP_EINVAL, "NULL argument");
    if (which < 0 || which > 2) return fail(MXP_EINVAL, "which must be 0 (exp), 1 (psi_1) or 2 (psi_2)");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    DeviceGuard guard(P->device);
    CKS(ensure_base(P));
    const int64_t ps = phi_dispatch(P, which, (const double2 *)x_dev, (double2 *)y_dev, 0);
    if (ps < 0) return MXP_ECUDA;
    CK(cudaGetLastError());
    CKS(read_scal(P, nullptr, 0));   // surfaces a persistent-kernel barrier timeout
    if (passes_out) *passes_out = ps;
    return MXP_OK;
}

mxp_status mxp_apply_matexpre(mxp_problem *P, const void *r_dev, void *w_dev, mxp_apply_stats *st)
{
    if (!P || !r_dev || !w_dev) return fail(MXP_EINVAL, "NULL argument");
    if (r_dev == w_dev) return fail(MXP_EINVAL, "r and w must not alias");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    DeviceGuard guard(P->device);
    return precond_apply(P, (const double2 *)r_dev, (double2 *)w_dev, st);
}

static mxp_status check_opts(const mxp_solve_opts *o)
{
    if (!o) return fail(MXP_EINVAL, "NULL options");
    if (!(o->rtol > 0) || !(o->rtol < 1)) return fail(MXP_EINVAL, "rtol must lie in (0, 1)");
    if (o->restart < 1 || o->restart > 64) return fail(MXP_EINVAL, "restart must lie in [1, 64]");
    if (o->maxit < 1) return fail(MXP_EINVAL, "maxit must be >= 1");
    return MXP_OK;
}

mxp_status mxp_solve(mxp_problem *P, const void *b_dev, void *x_dev, const mxp_solve_opts *opts,
                     mxp_solve_stats *st)
{
    if (!P || !b_dev || !x_dev) return fail(MXP_EINVAL, "NULL argument");
    if (b_dev == x_dev) return fail(MXP_EINVAL, "b and x must not alias");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    CKS(check_opts(opts));
    DeviceGuard guard(P->device);
    return fgmres_solve(P, (const double2 *)b_dev, (double2 *)x_dev, opts, st);
}

mxp_status mxp_solve_host(mxp_problem *P, const void *b_host, void *x_host, const mxp_solve_opts *opts,
                          mxp_solve_stats *st)
{
    if (!P || !b_host || !x_host) return fail(MXP_EINVAL, "NULL argument");
    if (P->slab) return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    CKS(check_opts(opts));
    DeviceGuard guard(P->device);
    const size_t bytes = (size_t)P->ntot * sizeof(double2);
    if (!P->bdev) CK(cudaMalloc(&P->bdev, bytes));
    if (!P->xdev) CK(cudaMalloc(&P->xdev, bytes));
    CK(cudaMemcpyAsync(P->bdev, b_host, bytes, cudaMemcpyHostToDevice, P->stream));
    if (opts->x0_given) CK(cudaMemcpyAsync(P->xdev, x_host, bytes, cudaMemcpyHostToDevice, P->stream));
    mxp_status s = fgmres_solve(P, P->bdev, P->xdev, opts, st);
    if (s != MXP_OK && s != MXP_ENOCONV) return s;
    CK(cudaMemcpyAsync(x_host, P->xdev, bytes, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return s;
}

mxp_status mxp_solve_batch(mxp_problem *const *probs, int nprob, int nrhs, const int *prob_of_rhs,
                           const void *const *b_dev, void *const *x_dev, const mxp_solve_opts *opts,
                           mxp_solve_stats *per_rhs)
{
    if (!probs || nprob < 1 || nrhs < 0 || (nrhs > 0 && (!prob_of_rhs || !b_dev || !x_dev)))
        return fail(MXP_EINVAL, "invalid batch arguments");
    CKS(check_opts(opts));
    for (int r = 0; r < nrhs; ++r)
        if (prob_of_rhs[r] < 0 || prob_of_rhs[r] >= nprob || !probs[prob_of_rhs[r]] || !b_dev[r] || !x_dev[r] ||
            b_dev[r] == x_dev[r])
            return fail(MXP_EINVAL, "invalid right-hand side entry");
    for (int q = 0; q < nprob; ++q)
        if (probs[q] && probs[q]->slab)
            return fail(MXP_EINVAL, "a slab problem runs mxp_horner_step and mxp_apply_operator only");
    // group the right-hand sides by problem handle (the same handle may appear twice)
    std::vector<mxp_problem *> handles;
    std::vector<std::vector<int>> groups;
    for (int r = 0; r < nrhs; ++r) {
        mxp_problem *P = probs[prob_of_rhs[r]];
        size_t gi = std::find(handles.begin(), handles.end(), P) - handles.begin();
        if (gi == handles.size()) {
            handles.push_back(P);
            groups.emplace_back();
        }
        groups[gi].push_back(r);
    }
    const size_t ng = groups.size();
    std::vector<mxp_status> status(ng, MXP_OK);
    std::vector<std::string> message(ng);
    std::vector<std::vector<mxp_solve_stats>> stats(ng);
    // A 2D problem that runs its exp actions on the persistent kernel and has at
    // least kSequentialUnknowns unknowns solves its sources one after another
    // (the single-source FGMRES, whose persistent launches fill the GPU and whose
    // inner GMRES restarts): on 1088^2 that is faster than the lockstep batch
    // (8 sources: 12.3 s against 19.4 s), which keeps every source until the
    // slowest converges and caps the inner iterations; on 544^2 and smaller grids
    // the batch wins.  Problems that launch the persistent (cooperative) kernel
    // never run concurrently with other work of this call.
    constexpr int64_t kSequentialUnknowns = (int64_t)1 << 20;
    std::vector<char> seq(ng, 0), coop(ng, 0);
    for (size_t gi = 0; gi < ng; ++gi) {
        coop[gi] = handles[gi]->grid.dim == 2 && handles[gi]->persist_cfg >= 0;
        seq[gi] = coop[gi] && handles[gi]->ntot >= kSequentialUnknowns;
    }
    // problems that qualify (2D, one low precision, one device, no faces,
    // Algorithm 1) form one group whose sources advance in lockstep, every pass
    // one launch over all of them; the others run one host thread each
    std::vector<size_t> gsel;
    for (size_t gi = 0; gi < ng; ++gi)
        if (!seq[gi] && groupable(handles[gi]) &&
            (gsel.empty() || (handles[gi]->device == handles[gsel[0]]->device &&
                              handles[gi]->prm.prec == handles[gsel[0]]->prm.prec)))
            gsel.push_back(gi);
    if (gsel.size() < 2) gsel.clear();
    std::vector<char> in_group(ng, 0);
    for (size_t gi : gsel) in_group[gi] = 1;
    mxp_status group_status = MXP_OK;
    std::string group_message;
    std::vector<mxp_solve_stats> group_stats(nrhs > 0 ? nrhs : 1, mxp_solve_stats{});
    auto run_group = [&]() {
        std::vector<mxp_problem *> gp;
        std::vector<std::vector<int>> rof;
        for (size_t gi : gsel) {
            gp.push_back(handles[gi]);
            rof.push_back(groups[gi]);
        }
        DeviceGuard guard(gp[0]->device);
        group_status = (gp[0]->prm.prec == MXP_C64)
                           ? group_solve_t<float2>(gp, rof, b_dev, x_dev, opts, group_stats)
                           : group_solve_t<__nv_bfloat162>(gp, rof, b_dev, x_dev, opts, group_stats);
        if (group_status != MXP_OK) group_message = g_last_error;
    };
    auto run = [&](size_t gi) {
        mxp_problem *P = handles[gi];
        DeviceGuard guard(P->device);
        std::vector<const double2 *> bs;
        std::vector<double2 *> xs;
        for (int r : groups[gi]) {
            bs.push_back((const double2 *)b_dev[r]);
            xs.push_back((double2 *)x_dev[r]);
        }
        stats[gi].assign(groups[gi].size(), mxp_solve_stats{});
        status[gi] = batch_solve(P, (int)groups[gi].size(), bs.data(), xs.data(), opts, stats[gi].data());
        if (status[gi] != MXP_OK) message[gi] = g_last_error;
    };
    auto run_seq = [&](size_t gi) {
        mxp_problem *P = handles[gi];
        DeviceGuard guard(P->device);
        stats[gi].assign(groups[gi].size(), mxp_solve_stats{});
        for (size_t q = 0; q < groups[gi].size() && status[gi] == MXP_OK; ++q) {
            const int r = groups[gi][q];
            const mxp_status sr = fgmres_solve(P, (const double2 *)b_dev[r], (double2 *)x_dev[r], opts, &stats[gi][q]);
            if (sr == MXP_ENOCONV) continue;        // reported through its statistics; the others still run
            status[gi] = sr;
            if (sr != MXP_OK) message[gi] = g_last_error;
        }
        if (status[gi] == MXP_OK)
            for (const mxp_solve_stats &q : stats[gi])
                if (!q.converged) status[gi] = MXP_ENOCONV;
    };
    // the group and the remaining problems run concurrently, one host thread
    // each (their kernels overlap on the GPU when they use different streams);
    // problems on the persistent kernel run afterwards, one at a time
    {
        std::vector<std::thread> th;
        if (!gsel.empty()) th.emplace_back(run_group);
        for (size_t gi = 0; gi < ng; ++gi)
            if (!in_group[gi] && !coop[gi]) th.emplace_back(run, gi);
        for (auto &t : th) t.join();
    }
    for (size_t gi = 0; gi < ng; ++gi) {
        if (in_group[gi] || !coop[gi]) continue;
        if (seq[gi]) run_seq(gi);
        else run(gi);
    }
    mxp_status worst = MXP_OK;
    if (!gsel.empty()) {
        if (per_rhs)
            for (size_t gi : gsel)
                for (int r : groups[gi]) per_rhs[r] = group_stats[r];
        if (group_status != MXP_OK && group_status != MXP_ENOCONV) return fail(group_status, group_message);
        if (group_status == MXP_ENOCONV) worst = MXP_ENOCONV;
    }
    for (size_t gi = 0; gi < ng; ++gi) {
        if (in_group[gi]) continue;
        if (per_rhs)
            for (size_t q = 0; q < groups[gi].size(); ++q) per_rhs[groups[gi][q]] = stats[gi][q];
        if (status[gi] != MXP_OK && status[gi] != MXP_ENOCONV) return fail(status[gi], message[gi]);
        if (status[gi] == MXP_ENOCONV) worst = MXP_ENOCONV;
    }
    if (worst == MXP_ENOCONV) return fail(MXP_ENOCONV, "a right-hand side did not converge");
    return MXP_OK;
}

void mxp_destroy(mxp_problem *P)
{
    if (!P) return;
    DeviceGuard guard(P->device);
    cudaStreamSynchronize(P->stream);
    cudaFree(P->c_dev); cudaFree(P->kappa64); cudaFree(P->kappa32);
    cudaFree(P->coef64); cudaFree(P->coef32); cudaFree(P->coef32s);
    cudaFree(P->face64); cudaFree(P->face32); cudaFree(P->face32s);
    for (int i = 0; i < 4; ++i) cudaFree(P->hb[i]);
    tma3_destroy(P->tma3);
    cudaFree(P->rt); cudaFree(P->tmp); cudaFree(P->tmp2); cudaFree(P->bdev); cudaFree(P->xdev);
    cudaFree(P->ks.partials);
    cudaFree(P->vec_dev);
    cudaFree(P->tau_dev);
    cudaFree(P->tau_psi_dev);
    cudaFree(P->wcoef_dev);
    cudaFree(P->bar);
    if (P->host_scal) cudaFreeHost(P->host_scal);
    free_arnoldi(P->inner);
    free_arnoldi(P->outer);
    free_batch(P);
    delete P;
}

}  // extern "C"
