// Fused 3D Taylor-Horner sweeps: K steps of one sub-step per launch by
// z-marching temporal blocking (Def. psi actions with the operator of
// Eq. pml-1d-s on each axis and the shift of Sec. 3.4).
//
// A CTA owns an x-y tile of (BX-2K) x (BY-2K) outputs and a segment of LZ
// planes along z.  It marches z upwards: each iteration loads one input plane
// (p, y, kappa) of the BX x BY region (tile plus K-cell halo) into a ring in
// shared memory, then level s = 1..K computes plane (iz - s) from level s-1's
// planes (iz - s - 1 .. iz - s + 1), and level K writes its plane to global
// memory.  One pass therefore reads p, y, kappa once and writes p once for K
// steps; x-y halo values become wrong by one cell per level and are never
// written.  Unknowns outside the grid stay zero (Dirichlet); tiles use the real
// interior coefficient 1/h^2 outside the PML.
#include <mutex>

#include "mxp_internal.h"

namespace mxp {

struct Fused3Scalars {
    float2 zfac;     // 1 + i s
    float ih2;       // 1 / h^2
    float tau[kMaxFuse];
    float2 rho;
    int rho_on;      // apply rho after the last step
};

template <typename S, int K, int BX, int BY>
__global__ void __launch_bounds__(BX *BY, 1) k_fused3d(Geom g, int LZ, const float2 *__restrict__ coef,
                                                       const float *__restrict__ kappa, Fused3Scalars sc,
                                                       const S *__restrict__ pin,
                                                       const S *__restrict__ yin,
                                                       S *__restrict__ pout)
{
    constexpr int PXW = BX + 2, PYH = BY + 2, PL = PXW * PYH;   // padded plane
    extern __shared__ float2 sm3[];
    float2 *Pr = sm3;                                 // [K][3][PYH][PXW] levels 0..K-1
    float2 *Yr = Pr + K * 3 * PL;                     // [K+1][PYH][PXW]
    float *Kr = reinterpret_cast<float *>(Yr + (K + 1) * PL);   // [K+1][BY][BX]

    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], nm = g.nmax;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int TX = BX - 2 * K, TY = BY - 2 * K;
    const int gx0 = blockIdx.x * TX - K, gy0 = blockIdx.y * TY - K;
    const int z0 = blockIdx.z * LZ, z1 = min(z0 + LZ, n2);
    const int gx = gx0 + tx, gy = gy0 + ty;
    const bool inxy = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
    const bool outxy = inxy && tx >= K && tx < K + TX && ty >= K && ty < K + TY;
    const int p0 = g.npml;
    const bool xyin = g.fast && gx >= p0 && gx < n0 - p0 && gy >= p0 && gy < n1 - p0;
    float2 wpx = make_float2(0.f, 0.f), wmx = wpx, wcx = wpx, wpy = wpx, wmy = wpx, wcy = wpx;
    if (inxy) {
        wpx = coef[gx]; wmx = coef[nm + gx]; wcx = coef[2 * nm + gx];
        wpy = coef[3 * nm + gy]; wmy = coef[4 * nm + gy]; wcy = coef[5 * nm + gy];
    }
    const float2 wcxy = make_float2(wcx.x + wcy.x, wcx.y + wcy.y);
    // zero every plane once (borders stay zero; out-of-grid cells are never written)
    for (int i = threadIdx.x; i < (K * 3 + K + 1) * PL; i += BX * BY) sm3[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int cell = (ty + 1) * PXW + tx + 1;
    const int64_t plane = (int64_t)n0 * n1;
    const int64_t qxy = (int64_t)gy * n0 + gx;

    // prefetch of the first input plane
    int iz = z0 - K;
    float2 np_ = make_float2(0.f, 0.f), ny_ = np_;
    float nk_ = 0.f;
    if (inxy && iz >= 0 && iz < n2) {
        np_ = St<S>::ld(pin, iz * plane + qxy);
        ny_ = St<S>::ld(yin, iz * plane + qxy);
        nk_ = kappa[iz * plane + qxy];
    }
    for (; iz < z1 + K; ++iz) {
        // level 0: the prefetched plane iz enters the rings
        Pr[(iz + 3 * K) % 3 * PL + cell] = np_;
        Yr[(iz + 3 * K) % (K + 1) * PL + cell] = ny_;
        Kr[(iz + 3 * K) % (K + 1) * BX * BY + ty * BX + tx] = nk_;
        // prefetch plane iz + 1 while the levels below compute
        const int jz = iz + 1;
        np_ = make_float2(0.f, 0.f);
        ny_ = np_;
        nk_ = 0.f;
        if (inxy && jz >= 0 && jz < n2 && jz < z1 + K) {
            np_ = St<S>::ld(pin, jz * plane + qxy);
            ny_ = St<S>::ld(yin, jz * plane + qxy);
            nk_ = kappa[jz * plane + qxy];
        }
        __syncthreads();
#pragma unroll
        for (int s = 1; s <= K; ++s) {
            const int z = iz - s;                    // plane produced by level s
            const bool valid = z >= z0 - K + s;      // its three input planes exist
            if (valid) {
                const float2 *src = Pr + (s - 1) * 3 * PL;
                const float2 *cm = src + (z + 3 * K - 1) % 3 * PL;
                const float2 *cc = src + (z + 3 * K) % 3 * PL;
                const float2 *cp = src + (z + 3 * K + 1) % 3 * PL;
                const bool in = inxy && z >= 0 && z < n2;
                float2 o = make_float2(0.f, 0.f);
                if (in) {
                    const float2 c = cc[cell];
                    const float2 e = cc[cell + 1], w = cc[cell - 1];
                    const float2 nth = cc[cell + PXW], sth = cc[cell - PXW];
                    const float2 up = cp[cell], dn = cm[cell];
                    const float2 wpz = coef[6 * nm + z], wmz = coef[7 * nm + z], wcz = coef[8 * nm + z];
                    float2 q;
                    if (xyin && z >= p0 && z < n2 - p0) {
                        q.x = (e.x + w.x + nth.x + sth.x + up.x + dn.x) * sc.ih2;
                        q.y = (e.y + w.y + nth.y + sth.y + up.y + dn.y) * sc.ih2;
                    } else {
                        q = cadd(cadd(cadd(cmul(wpx, e), cmul(wmx, w)), cadd(cmul(wpy, nth), cmul(wmy, sth))),
                                 cadd(cmul(wpz, up), cmul(wmz, dn)));
                    }
                    const float kp = Kr[(z + 3 * K) % (K + 1) * BX * BY + ty * BX + tx];
                    // diagonal kappa (1 + i s) - sum_d wc_d (mu folded in the wc rows)
                    const float2 d = make_float2(kp * sc.zfac.x - wcxy.x - wcz.x, kp * sc.zfac.y - wcxy.y - wcz.y);
                    q = cadd(q, cmul(d, c));
                    const float2 yv = Yr[(z + 3 * K) % (K + 1) * PL + cell];
                    const float tau = sc.tau[s - 1];
                    o = make_float2(yv.x - tau * q.y, yv.y + tau * q.x);
                    if (s == K && sc.rho_on) o = cmul(sc.rho, o);
                }
                if (s < K) {
                    Pr[s * 3 * PL + (z + 3 * K) % 3 * PL + cell] = o;
                } else if (outxy && z >= z0 && z < z1) {
                    St<S>::st(pout, z * plane + qxy, o);
                }
            }
            __syncthreads();
        }
    }
}

struct Tile3 {
    int K, BX, BY;
};
static const Tile3 kT3[] = {{2, 64, 16}, {2, 32, 32}, {4, 32, 32}, {4, 64, 16}};
constexpr int kNumT3 = sizeof(kT3) / sizeof(kT3[0]);

int fused3d_num_cfgs() { return kNumT3; }
int fused3d_cfg_k(int id) { return kT3[id].K; }

template <typename S, int K, int BX, int BY>
static void launch3(const Geom &g, int lz, const float2 *coef, const float *kappa, const Fused3Scalars &sc,
                    const S *pin, const S *y, S *pout, cudaStream_t st)
{
    constexpr int PL = (BX + 2) * (BY + 2);
    const size_t smem = (size_t)(K * 3 + K + 1) * PL * sizeof(float2) + (size_t)(K + 1) * BX * BY * sizeof(float);
    // opt in to large dynamic shared memory once per device (per template instance)
    static std::atomic<bool> configured[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev].load()) {
        cudaFuncSetAttribute(k_fused3d<S, K, BX, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured[dev].store(true);
    }
    dim3 grid((g.n[0] + BX - 2 * K - 1) / (BX - 2 * K), (g.n[1] + BY - 2 * K - 1) / (BY - 2 * K),
              (g.n[2] + lz - 1) / lz);
    count_launch();
    k_fused3d<S, K, BX, BY><<<grid, BX * BY, smem, st>>>(g, lz, coef, kappa, sc, pin, y, pout);
}

template <typename S>
bool launch_fused3d(int cfg, int lz, const Geom &g, const float2 *coef, const float *kappa,
                    const FusedStep *steps, float2 zfac, const S *pin, const S *y, S *pout, cudaStream_t st)
{
    if (g.dim != 3 || cfg < 0 || cfg >= kNumT3) return false;
    Fused3Scalars sc;
    sc.zfac = zfac;
    sc.ih2 = (float)g.ih2;
    sc.rho = make_float2(1.f, 0.f);
    sc.rho_on = 0;
    const int K = kT3[cfg].K;
    for (int s = 0; s < K; ++s) {
        sc.tau[s] = (float)steps[s].tau;
        if (steps[s].rho_on) {
            sc.rho = make_float2((float)steps[s].rho_re, (float)steps[s].rho_im);
            sc.rho_on = 1;
        }
    }
    if (lz < 1) lz = 64;
    switch (cfg) {
    case 0: launch3<S, 2, 64, 16>(g, lz, coef, kappa, sc, pin, y, pout, st); break;
    case 1: launch3<S, 2, 32, 32>(g, lz, coef, kappa, sc, pin, y, pout, st); break;
    case 2: launch3<S, 4, 32, 32>(g, lz, coef, kappa, sc, pin, y, pout, st); break;
    default: launch3<S, 4, 64, 16>(g, lz, coef, kappa, sc, pin, y, pout, st); break;
    }
    return true;
}

template bool launch_fused3d<float2>(int, int, const Geom &, const float2 *, const float *, const FusedStep *,
                                     float2, const float2 *, const float2 *, float2 *, cudaStream_t);
template bool launch_fused3d<__nv_bfloat162>(int, int, const Geom &, const float2 *, const float *,
                                             const FusedStep *, float2, const __nv_bfloat162 *,
                                             const __nv_bfloat162 *, __nv_bfloat162 *, cudaStream_t);

}  // namespace mxp
