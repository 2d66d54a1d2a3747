// Fused 2D Taylor-Horner sweeps: K consecutive steps of one sub-step per launch
// (temporal blocking).  Step s computes
//     p <- rho_s ( y + i tau_s (A_s - mu) p + gamma_s v )
// with the PML operator of Eq. pml-1d-s (per-axis coefficient table) and the
// complex shift of Sec. 3.4.  Each CTA loads a region of RX x RY unknowns
// (its output tile plus a K-cell halo on every side) into shared memory, runs
// the K steps there, and writes back the inner (RX-2K) x (RY-2K) tile, so one
// pass reads p, y, kappa (and v) and writes p once for K steps.
//
// Thread layout: RX lanes along x (coalesced rows), G groups of RT consecutive
// rows; a thread walks its RT rows keeping the north/centre/south values in
// registers, so each step costs one shared load down the column plus the two
// x-neighbours.  y, v and the per-point diagonal live in registers for the
// whole pass.  Values at region edges are wrong after a step but the error
// moves in by one cell per step, so after K steps the inner tile is exact.
// Unknowns outside the grid are forced to zero (Dirichlet) at every step.
// Tiles whose region avoids the PML use the real interior coefficients 1/h^2.
#include <mutex>

#include "mxp_internal.h"

namespace mxp {

// One tile (bxi, byi) of one vector: the body shared by the single-grid kernel
// and the grouped kernel.  sm: dynamic shared memory of the block.
template <typename S, int K, int RX, int RT, int G, bool HAS_V>
__device__ __forceinline__ void fused2d_tile(int n0, int n1, int npml, int nmax, int TXO, int TYO, int bxi,
                                             int byi, const float2 *__restrict__ coef,
                                             const float *__restrict__ kappa, const FusedScalars &sc,
                                             const S *__restrict__ pin, const S *__restrict__ yv_g,
                                             const S *__restrict__ v_g, S *__restrict__ pout, float2 *sm)
{
    constexpr int RY = RT * G;
    constexpr int PX = RX + 2;                 // padded row (zero column on each side)
    // output tile TXO x TYO (<= RX-2K x RY-2K, chosen at run time); region = tile + K halo
    float2 *buf0 = sm;
    float2 *buf1 = sm + (RY + 2) * PX;
    float2 *cy = buf1 + (RY + 2) * PX;         // [RY][2]: wp_y, wm_y of each region row

    const int tx = threadIdx.x % RX;
    const int grp = threadIdx.x / RX;
    const int gx0 = bxi * TXO - K;
    const int gy0 = byi * TYO - K;
    const int gx = gx0 + tx;
    const bool inx = (gx >= 0) && (gx < n0);
    const bool interior = (gx0 >= npml) && (gx0 + TXO + 2 * K <= n0 - npml) && (gy0 >= npml) &&
                          (gy0 + TYO + 2 * K <= n1 - npml);

    // zero the padding frame of both buffers
    for (int i = threadIdx.x; i < 2 * (RY + 2); i += RX * G) {
        const int b = i / (RY + 2), r = i % (RY + 2);
        float2 *buf = b ? buf1 : buf0;
        buf[r * PX] = make_float2(0.f, 0.f);
        buf[r * PX + RX + 1] = make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < 2 * RX; i += RX * G) {
        const int b = i / RX, c = i % RX;
        float2 *buf = b ? buf1 : buf0;
        buf[c + 1] = make_float2(0.f, 0.f);
        buf[(RY + 1) * PX + c + 1] = make_float2(0.f, 0.f);
    }
    // y-axis coefficients of the region rows
    for (int r = threadIdx.x; r < RY; r += RX * G) {
        const int gy = gy0 + r;
        float2 wp = make_float2(0.f, 0.f), wm = make_float2(0.f, 0.f);
        if (gy >= 0 && gy < n1) {
            wp = coef[3 * nmax + gy];
            wm = coef[4 * nmax + gy];
        }
        cy[2 * r] = wp;
        cy[2 * r + 1] = wm;
    }
    float2 wpx = make_float2(0.f, 0.f), wmx = make_float2(0.f, 0.f), wcx = make_float2(0.f, 0.f);
    if (inx) {
        wpx = coef[gx];
        wmx = coef[nmax + gx];
        wcx = coef[2 * nmax + gx];
    }

    float2 yr[RT], dr[RT];
    float2 vr[HAS_V ? RT : 1];
    float2 pr[RT];
    float kr[RT];
    float2 wcyr[RT];
    unsigned mask = 0u;
    // issue every global load of this thread first (clamped, always-valid
    // addresses), then mask: many loads in flight instead of one per row
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int gy = gy0 + grp * RT + r;
        const bool in = inx && (gy >= 0) && (gy < n1);
        if (in) mask |= 1u << r;
        const int64_t q = in ? (int64_t)gy * n0 + gx : 0;
        const int gyc = (gy < 0) ? 0 : ((gy >= n1) ? n1 - 1 : gy);
        pr[r] = St<S>::ld(pin, q);
        yr[r] = St<S>::ld(yv_g, q);
        kr[r] = kappa[q];
        wcyr[r] = coef[5 * nmax + gyc];
        if (HAS_V) vr[HAS_V ? r : 0] = St<S>::ld(v_g, q);
    }
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int ry = grp * RT + r;
        const bool in = (mask >> r) & 1u;
        const float2 zero = make_float2(0.f, 0.f);
        buf0[(ry + 1) * PX + tx + 1] = in ? pr[r] : zero;
        yr[r] = in ? yr[r] : zero;
        if (HAS_V) vr[HAS_V ? r : 0] = in ? vr[HAS_V ? r : 0] : zero;
        dr[r] = in ? make_float2(kr[r] * sc.zfac.x - sc.mu - wcx.x - wcyr[r].x,
                                 kr[r] * sc.zfac.y - wcx.y - wcyr[r].y)
                   : zero;
    }
    __syncthreads();

#pragma unroll 1
    for (int s = 0; s < K; ++s) {
        const float2 *src = (s & 1) ? buf1 : buf0;
        float2 *dst = (s & 1) ? buf0 : buf1;
        const float tau = sc.tau[s];
        const float2 gam = sc.gamma[s];
        const bool last_rho = (s == K - 1) && sc.rho_on;
        const int r0 = grp * RT;                // first region row of this thread
        float2 up = src[r0 * PX + tx + 1];
        float2 cen = src[(r0 + 1) * PX + tx + 1];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int ry = r0 + r;
            const float2 dn = src[(ry + 2) * PX + tx + 1];
            const float2 e = src[(ry + 1) * PX + tx + 2];
            const float2 w = src[(ry + 1) * PX + tx];
            float2 q;
            if (interior) {
                q.x = (e.x + w.x + up.x + dn.x) * sc.ih2;
                q.y = (e.y + w.y + up.y + dn.y) * sc.ih2;
            } else {
                const float2 wpy = cy[2 * ry], wmy = cy[2 * ry + 1];
                q = cadd(cadd(cmul(wpx, e), cmul(wmx, w)), cadd(cmul(wpy, dn), cmul(wmy, up)));
            }
            q = cadd(q, cmul(dr[r], cen));
            float2 o = make_float2(yr[r].x - tau * q.y, yr[r].y + tau * q.x);
            if (HAS_V) o = cadd(o, cmul(gam, vr[HAS_V ? r : 0]));
            if (last_rho) o = cmul(sc.rho, o);
            if (!((mask >> r) & 1u)) o = make_float2(0.f, 0.f);
            dst[(ry + 1) * PX + tx + 1] = o;
            up = cen;
            cen = dn;
        }
        __syncthreads();
    }

    const float2 *fin = (K & 1) ? buf1 : buf0;
    if (tx >= K && tx < K + TXO) {
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int ry = grp * RT + r;
            if (ry >= K && ry < K + TYO && ((mask >> r) & 1u)) {
                const int64_t q = (int64_t)(gy0 + ry) * n0 + gx;
                St<S>::st(pout, q, fin[(ry + 1) * PX + tx + 1]);
            }
        }
    }
}

template <typename S, int K, int RX, int RT, int G, bool HAS_V>
__global__ void __launch_bounds__(RX *G, (RX * G <= 512 && !HAS_V) ? 2 : 1) k_fused2d(int n0, int n1, int npml, int nmax, int TXO,
                                                   int TYO,
                                                   const float2 *__restrict__ coef,
                                                   const float *__restrict__ kappa,
                                                   const FusedScalars sc,
                                                   const S *__restrict__ pin,
                                                   const S *__restrict__ yv_g,
                                                   const S *__restrict__ v_g,
                                                   S *__restrict__ pout)
{
    extern __shared__ float2 sm[];
    // blockIdx.z selects one vector of a batch (vectors of one grid, n0*n1 apart)
    const int64_t off = (int64_t)blockIdx.z * n0 * n1;
    fused2d_tile<S, K, RX, RT, G, HAS_V>(n0, n1, npml, nmax, TXO, TYO, blockIdx.x, blockIdx.y, coef, kappa, sc,
                                         pin + off, yv_g + off, HAS_V ? v_g + off : v_g, pout + off, sm);
}

// The same pass for a group of grids of different sizes in one launch: block b
// takes the work item bmap[b] = (problem, source of that problem, tile x, tile
// y); a block whose source has converged (active[source] == 0) returns at
// once, so one captured launch sequence serves every subset of live sources.
// The scalars of the pass differ per problem (t, the shift and the psi_1
// coefficients depend on the grid); slot indices select the problem's batch
// buffers (its sources' vectors n0 * n1 apart).
template <typename S, int K, int RX, int RT, int G, bool HAS_V>
__global__ void __launch_bounds__(RX *G, (RX * G <= 512 && !HAS_V) ? 2 : 1)
    k_fused2d_group(const GroupProblem *__restrict__ gp, const int4 *__restrict__ bmap,
                    const FusedScalars *__restrict__ sc_tab, const int *__restrict__ active, int iin, int iy,
                    int iv, int iout)
{
    extern __shared__ float2 sm[];
    const int4 m = bmap[blockIdx.x];
    const GroupProblem &P = gp[m.x];
    if (active[P.src0 + m.y] == 0) return;         // uniform over the block
    const int n0 = P.n0, n1 = P.n1;
    const int64_t off = (int64_t)m.y * n0 * n1;
    const S *pin = static_cast<const S *>(P.slot[iin]) + off;
    const S *yv = static_cast<const S *>(P.slot[iy]) + off;
    const S *v = HAS_V ? static_cast<const S *>(P.slot[iv]) + off : nullptr;
    S *pout = static_cast<S *>(P.slot[iout]) + off;
    const FusedScalars &sc = sc_tab[m.x];
    fused2d_tile<S, K, RX, RT, G, HAS_V>(n0, n1, P.npml, P.nmax, P.txo, P.tyo, m.z, m.w, P.coef, P.kappa, sc,
                                         pin, yv, v, pout, sm);
}

struct TileCfg {
    int K, RX, RT, G;
};

// Tile configurations the tuner may pick from (index = cfg id).
static const TileCfg kCfgs[] = {
    {2, 128, 8, 4}, {4, 128, 8, 4}, {8, 128, 8, 4}, {4, 64, 4, 8},
    {2, 64, 4, 8},  {8, 128, 12, 4}, {4, 128, 4, 4}, {6, 128, 8, 4},
};
constexpr int kNumCfgs = sizeof(kCfgs) / sizeof(kCfgs[0]);

int fused2d_num_cfgs() { return kNumCfgs; }
int fused2d_cfg_k(int id) { return kCfgs[id].K; }

template <typename S, int K, int RX, int RT, int G, bool HAS_V>
static void launch_one(int n0, int n1, int npml, int nmax, int tyo, int nb, const float2 *coef,
                       const float *kappa, const FusedScalars &sc, const S *pin, const S *y,
                       const S *v, S *pout, cudaStream_t st)
{
    constexpr int RY = RT * G;
    const size_t smem = (size_t)(2 * (RY + 2) * (RX + 2) + 2 * RY) * sizeof(float2);
    // opt in to large dynamic shared memory once per device (per template instance)
    static std::atomic<bool> configured[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev].load()) {
        cudaFuncSetAttribute(k_fused2d<S, K, RX, RT, G, HAS_V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured[dev].store(true);
    }
    // balance the x tiles: ceil(n0 / (RX-2K)) tiles of equal width
    const int ntx = (n0 + RX - 2 * K - 1) / (RX - 2 * K);
    const int txo = (n0 + ntx - 1) / ntx;
    if (tyo <= 0 || tyo > RY - 2 * K) tyo = RY - 2 * K;
    dim3 grid(ntx, (n1 + tyo - 1) / tyo, nb);
    count_launch();
    k_fused2d<S, K, RX, RT, G, HAS_V><<<grid, RX * G, smem, st>>>(n0, n1, npml, nmax, txo, tyo,
                                                                 coef, kappa, sc, pin, y, v, pout);
}

template <typename S, int K, int RX, int RT, int G>
static void launch_v(bool hv, int n0, int n1, int npml, int nmax, int tyo, int nb,
                     const float2 *coef, const float *kappa, const FusedScalars &sc, const S *pin,
                     const S *y, const S *v, S *pout, cudaStream_t st)
{
    if (hv) launch_one<S, K, RX, RT, G, true>(n0, n1, npml, nmax, tyo, nb, coef, kappa, sc, pin, y, v, pout, st);
    else launch_one<S, K, RX, RT, G, false>(n0, n1, npml, nmax, tyo, nb, coef, kappa, sc, pin, y, v, pout, st);
}

int fused2d_cfg_rx(int id) { return kCfgs[id].RX; }
int fused2d_cfg_max_tyo(int id) { return kCfgs[id].RT * kCfgs[id].G - 2 * kCfgs[id].K; }

template <typename S>
bool launch_fused2d(int cfg, int tyo, const Geom &g, int npml, const float2 *coef, const float *kappa,
                    const FusedStep *steps, const float2 zfac, float mu, float ih2,
                    const S *pin, const S *y, const S *v, S *pout, cudaStream_t st, int nb)
{
    if (g.dim != 2 || cfg < 0 || cfg >= kNumCfgs) return false;
    FusedScalars sc;
    sc.zfac = zfac;
    sc.mu = mu;
    sc.ih2 = ih2;
    const int K = kCfgs[cfg].K;
    sc.rho = make_float2(1.f, 0.f);
    sc.rho_on = 0;
    for (int s = 0; s < K; ++s) {
        sc.tau[s] = (float)steps[s].tau;
        sc.gamma[s] = make_float2((float)steps[s].gamma_re, (float)steps[s].gamma_im);
        if (steps[s].rho_on) {
            sc.rho = make_float2((float)steps[s].rho_re, (float)steps[s].rho_im);
            sc.rho_on = 1;
        }
    }
    const bool hv = (v != nullptr);
    const int n0 = g.n[0], n1 = g.n[1], nm = g.nmax;
    switch (cfg) {
    case 0: launch_v<S, 2, 128, 8, 4>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 1: launch_v<S, 4, 128, 8, 4>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 2: launch_v<S, 8, 128, 8, 4>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 3: launch_v<S, 4, 64, 4, 8>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 4: launch_v<S, 2, 64, 4, 8>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 5: launch_v<S, 8, 128, 12, 4>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 6: launch_v<S, 4, 128, 4, 4>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    case 7: launch_v<S, 6, 128, 8, 4>(hv, n0, n1, npml, nm, tyo, nb, coef, kappa, sc, pin, y, v, pout, st); break;
    default: return false;
    }
    return true;
}

void fused2d_scalars(int cfg, const FusedStep *steps, float2 zfac, float mu, float ih2, FusedScalars *out)
{
    FusedScalars &sc = *out;
    sc.zfac = zfac;
    sc.mu = mu;
    sc.ih2 = ih2;
    sc.rho = make_float2(1.f, 0.f);
    sc.rho_on = 0;
    const int K = kCfgs[cfg].K;
    for (int s = 0; s < kMaxFuse; ++s) {
        sc.tau[s] = 0.f;
        sc.gamma[s] = make_float2(0.f, 0.f);
    }
    for (int s = 0; s < K; ++s) {
        sc.tau[s] = (float)steps[s].tau;
        sc.gamma[s] = make_float2((float)steps[s].gamma_re, (float)steps[s].gamma_im);
        if (steps[s].rho_on) {
            sc.rho = make_float2((float)steps[s].rho_re, (float)steps[s].rho_im);
            sc.rho_on = 1;
        }
    }
}

bool fused2d_tiles(int cfg, int n0, int n1, int tyo, int *txo, int *tyo_out, int *ntx, int *nty)
{
    if (cfg < 0 || cfg >= kNumCfgs || n0 < 1 || n1 < 1) return false;
    const TileCfg c = kCfgs[cfg];
    const int RY = c.RT * c.G;
    *ntx = (n0 + c.RX - 2 * c.K - 1) / (c.RX - 2 * c.K);
    *txo = (n0 + *ntx - 1) / *ntx;
    if (tyo <= 0 || tyo > RY - 2 * c.K) tyo = RY - 2 * c.K;
    *tyo_out = tyo;
    *nty = (n1 + tyo - 1) / tyo;
    return true;
}

template <typename S, int K, int RX, int RT, int G, bool HAS_V>
static void launch_group_one(const GroupProblem *gp, const int4 *bmap, int nblocks, const FusedScalars *sc_tab,
                             const int *active, int iin, int iy, int iv, int iout, cudaStream_t st)
{
    constexpr int RY = RT * G;
    const size_t smem = (size_t)(2 * (RY + 2) * (RX + 2) + 2 * RY) * sizeof(float2);
    static std::atomic<bool> configured[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev].load()) {
        cudaFuncSetAttribute(k_fused2d_group<S, K, RX, RT, G, HAS_V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        configured[dev].store(true);
    }
    count_launch();
    k_fused2d_group<S, K, RX, RT, G, HAS_V><<<nblocks, RX * G, smem, st>>>(gp, bmap, sc_tab, active, iin, iy, iv,
                                                                          iout);
}

template <typename S, int K, int RX, int RT, int G>
static void launch_group_v(bool hv, const GroupProblem *gp, const int4 *bmap, int nblocks,
                           const FusedScalars *sc_tab, const int *active, int iin, int iy, int iv, int iout,
                           cudaStream_t st)
{
    if (hv) launch_group_one<S, K, RX, RT, G, true>(gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st);
    else launch_group_one<S, K, RX, RT, G, false>(gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st);
}

template <typename S>
bool launch_fused2d_group(int cfg, const GroupProblem *gp, const int4 *bmap, int nblocks,
                          const FusedScalars *sc_tab, const int *active, int iin, int iy, int iv, int iout,
                          cudaStream_t st)
{
    if (cfg < 0 || cfg >= kNumCfgs || nblocks < 1) return false;
    const bool hv = iv >= 0;
    if (!hv) iv = 0;
    switch (cfg) {
    case 0: launch_group_v<S, 2, 128, 8, 4>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 1: launch_group_v<S, 4, 128, 8, 4>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 2: launch_group_v<S, 8, 128, 8, 4>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 3: launch_group_v<S, 4, 64, 4, 8>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 4: launch_group_v<S, 2, 64, 4, 8>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 5: launch_group_v<S, 8, 128, 12, 4>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 6: launch_group_v<S, 4, 128, 4, 4>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    case 7: launch_group_v<S, 6, 128, 8, 4>(hv, gp, bmap, nblocks, sc_tab, active, iin, iy, iv, iout, st); break;
    default: return false;
    }
    return true;
}

template bool launch_fused2d_group<float2>(int, const GroupProblem *, const int4 *, int, const FusedScalars *,
                                           const int *, int, int, int, int, cudaStream_t);
template bool launch_fused2d_group<__nv_bfloat162>(int, const GroupProblem *, const int4 *, int,
                                                   const FusedScalars *, const int *, int, int, int, int,
                                                   cudaStream_t);

template bool launch_fused2d<float2>(int, int, const Geom &, int, const float2 *, const float *,
                                     const FusedStep *, const float2, float, float, const float2 *,
                                     const float2 *, const float2 *, float2 *, cudaStream_t, int);
template bool launch_fused2d<__nv_bfloat162>(int, int, const Geom &, int, const float2 *, const float *,
                                             const FusedStep *, const float2, float, float,
                                             const __nv_bfloat162 *, const __nv_bfloat162 *,
                                             const __nv_bfloat162 *, __nv_bfloat162 *, cudaStream_t, int);

}  // namespace mxp
