// 3D Taylor-Horner sweep (one step of the exp / psi actions of Def. psi on the
// operator of Eq. helmholtz, Eq. pml-1d-s and Sec. 3.4) with the planes staged
// in shared memory by the Tensor Memory Accelerator.
//
// A block of 32 x 8 threads owns a 32 x 16 column of the grid (two rows per
// thread, which halves the per-plane barriers and waits per point) over a
// segment of planes and marches along z.  Plane z of p (the tile plus a halo), of y, of kappa and of v is
// brought into one stage of a ring in shared memory by cp.async.bulk.tensor
// loads that one thread issues several planes ahead; an mbarrier per stage
// counts the bytes that arrived.  The step at plane z then reads p(z-1), p(z),
// p(z+1) and the x / y neighbours from shared memory only, so the SM keeps many
// planes in flight without holding them in registers, and DRAM sees the
// compulsory bytes of every point once.  TMA fills cells outside the grid with
// zeros, which is the zero Dirichlet condition.
//
// Alignment: a tiled TMA load must start at a 16-byte boundary in x.  Vectors
// are viewed as arrays of 4-byte elements (a complex64 value is two of them, a
// bf16x2 value one), the tile starts at x0 (a multiple of 32) and its left halo
// is widened to 2 (complex64) or 4 (bf16x2) cells, so every x start is a
// multiple of 16 bytes.  Row strides must be multiples of 16 bytes, which holds
// when n0 is a multiple of 4; other grids use the register-marching sweep.
//
// Every wait on an mbarrier is bounded: on timeout the kernel sets the error
// word (reported as MXP_ETIMEOUT), stops issuing loads, waits (again bounded) for
// the loads it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mxp_internal.h"

#ifndef MXP_TMA3_STAGES
#define MXP_TMA3_STAGES 6
#endif
#ifndef MXP_TMA3_RPT
#define MXP_TMA3_RPT 2
#endif

namespace mxp {

constexpr int kRPT = MXP_TMA3_RPT;        // rows of the tile per thread
constexpr int kTX = 32, kTY = 8 * kRPT;   // tile of a block (32 x 8 threads)
constexpr int kStages = MXP_TMA3_STAGES;  // planes resident or in flight per block
constexpr long long kTmaPollLimit = 1ll << 22;

template <typename S> struct TmaElt;
template <> struct TmaElt<float2> {        // complex64: two 4-byte elements per value
    static constexpr int E = 2, HL = 2;
};
template <> struct TmaElt<__nv_bfloat162> {  // bf16x2: one 4-byte element per value
    static constexpr int E = 1, HL = 4;
};

template <typename S> struct Tma3Geo {
    static constexpr int PW = kTX + 2 * TmaElt<S>::HL;   // p tile row, in values
    static constexpr int PBYTES = (kTY + 2) * PW * (int)sizeof(S);
    static constexpr int YBYTES = kTY * kTX * (int)sizeof(S);
    static constexpr int KBYTES = kTY * kTX * 4;
    static constexpr int al(int b) { return (b + 127) / 128 * 128; }
    static constexpr int stage_bytes(bool has_y, bool has_v)
    {
        return al(PBYTES) + (has_y ? al(YBYTES) : 0) + al(KBYTES) + (has_v ? al(YBYTES) : 0);
    }
    static constexpr int tx_bytes(bool has_y, bool has_v)
    {
        return PBYTES + (has_y ? YBYTES : 0) + KBYTES + (has_v ? YBYTES : 0);
    }
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                          unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        :
        : "r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
          "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed; false after the limit
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (long long it = 0; it < kTmaPollLimit; ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename C>
__device__ __forceinline__ C czero3() { return CT<C>::mk(0, 0); }

template <typename S>
__device__ __forceinline__ typename St<S>::C sm_ld(const S *p, int i)
{
    return St<S>::ld(p, i);
}

template <typename S, bool HAS_Y, bool HAS_V>
__global__ void __launch_bounds__(kTX * 8) k_step3z_tma(Geom g, const typename St<S>::C *__restrict__ coef,
                                                         StepScalars<typename St<S>::C> sc,
                                                         const __grid_constant__ CUtensorMap mp,
                                                         const __grid_constant__ CUtensorMap my,
                                                         const __grid_constant__ CUtensorMap mk,
                                                         const __grid_constant__ CUtensorMap mv,
                                                         S *__restrict__ pout, int lz, unsigned *err)
{
    using C = typename St<S>::C;
    using R = typename St<S>::R;
    using G = Tma3Geo<S>;
    constexpr int HL = TmaElt<S>::HL, E = TmaElt<S>::E, PW = G::PW;
    constexpr int SB = G::stage_bytes(HAS_Y, HAS_V);
    constexpr unsigned TXB = (unsigned)G::tx_bytes(HAS_Y, HAS_V);
    extern __shared__ __align__(128) unsigned char stg_raw[];
    __shared__ __align__(8) unsigned long long bar[kStages];
    __shared__ int s_fail;
    // TMA destinations start at 128-byte boundaries (the launch adds 128 bytes of slack)
    unsigned char *stg = stg_raw + ((128u - (smem_u32(stg_raw) & 127u)) & 127u);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], nm = g.nmax;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int z0 = blockIdx.z * lz, z1 = min(z0 + lz, n2);
    const int i = x0 + tx;          // rows of this thread: y0 + ty + 8 rr, rr < kRPT
    const int nplanes = z1 - z0 + 2;          // planes z0-1 .. z1

    // byte offsets of the parts of a stage
    constexpr int OY = G::al(G::PBYTES);
    constexpr int OK = OY + (HAS_Y ? G::al(G::YBYTES) : 0);
    constexpr int OV = OK + G::al(G::KBYTES);
    // plane index pi (0 .. nplanes-1) is plane z0 - 1 + pi, held by stage pi % kStages;
    // stage numbers and mbarrier parities advance incrementally
    auto issue = [&](int pi, int st) {
        const int z = z0 - 1 + pi;
        unsigned char *b = stg + st * SB;
        mbar_expect(&bar[st], TXB);
        tma_load3(b, &mp, E * (x0 - HL), y0 - 1, z, &bar[st]);
        if (HAS_Y) tma_load3(b + OY, &my, E * x0, y0, z, &bar[st]);
        tma_load3(b + OK, &mk, x0, y0, z, &bar[st]);
        if (HAS_V) tma_load3(b + OV, &mv, E * x0, y0, z, &bar[st]);
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();
    // producer / waiter state, used by thread 0 only
    int issued = 0, is_stage = 0;             // next plane to load and its stage
    int waited = -1, w_stage = 0, w_par = 0;  // planes 0 .. waited resident; next stage to wait on
    if (tid == 0) {
        for (; issued < kStages && issued < nplanes; ++issued) {
            issue(issued, is_stage);
            if (++is_stage == kStages) is_stage = 0;
        }
    }

    // per-column coefficients (constant along z)
    const C *cz = coef + 6 * nm;
    const int p0 = g.npml;
    C wpx = czero3<C>(), wmx = wpx, wcx = wpx;
    if (i < n0) { wpx = coef[i]; wmx = coef[nm + i]; wcx = coef[2 * nm + i]; }
    C wpy[kRPT], wmy[kRPT], wcy[kRPT];
    bool active[kRPT], xyin[kRPT];
#pragma unroll
    for (int rr = 0; rr < kRPT; ++rr) {
        const int j = y0 + ty + 8 * rr;
        active[rr] = i < n0 && j < n1;
        wpy[rr] = wmy[rr] = wcy[rr] = czero3<C>();
        if (active[rr]) { wpy[rr] = coef[3 * nm + j]; wmy[rr] = coef[4 * nm + j]; wcy[rr] = coef[5 * nm + j]; }
        xyin[rr] = g.fast && i >= p0 && i < n0 - p0 && j >= p0 && j < n1 - p0;
    }
    int sm_ = 0, sc_ = 1, sp_ = 2;            // stages of planes pi - 1, pi, pi + 1
    S *outp = pout + (i + g.s1 * (y0 + ty) + g.s2 * z0);
    // z-axis coefficients of the current plane, loaded one plane ahead
    C czp = cz[z0], czm = cz[nm + z0], czc = cz[2 * nm + z0];

    for (int k = z0; k < z1; ++k, outp += g.s2) {
        const int pi = k - z0 + 1;            // plane index of z = k
        // thread 0 waits until planes pi - 1, pi, pi + 1 are resident; the block
        // barrier then orders those TMA writes before every thread's reads
        if (tid == 0) {
            bool ok = true;
            while (waited < pi + 1) {
                ok = mbar_wait(&bar[w_stage], (unsigned)w_par);
                if (!ok) break;
                ++waited;
                if (++w_stage == kStages) { w_stage = 0; w_par ^= 1; }
            }
            if (!ok) {
                atomicExch(err, 1u);
                s_fail = 1;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const int kn = (k + 1 < n2) ? k + 1 : k;
        const C czp_n = cz[kn], czm_n = cz[nm + kn], czc_n = cz[2 * nm + kn];
        {
            const unsigned char *bc = stg + sc_ * SB;
            const S *pc_ = reinterpret_cast<const S *>(bc);
            const S *pm_ = reinterpret_cast<const S *>(stg + sm_ * SB);
            const S *pp_ = reinterpret_cast<const S *>(stg + sp_ * SB);
#pragma unroll
            for (int rr = 0; rr < kRPT; ++rr) {
                if (!active[rr]) continue;
                const int cidx = (ty + 8 * rr + 1) * PW + tx + HL;
                const int tidx = (ty + 8 * rr) * kTX + tx;
                const C pc = sm_ld<S>(pc_, cidx);
                const C xp = sm_ld<S>(pc_, cidx + 1), xm = sm_ld<S>(pc_, cidx - 1);
                const C yp = sm_ld<S>(pc_, cidx + PW), ym = sm_ld<S>(pc_, cidx - PW);
                const C pp = sm_ld<S>(pp_, cidx), pm = sm_ld<S>(pm_, cidx);
                const bool inner = xyin[rr] && k >= p0 && k < n2 - p0;
                C acc;
                if (inner) {
                    acc = cadd(cadd(cadd(xp, xm), cadd(yp, ym)), cadd(pp, pm));
                    const R s = (R)g.ih2;
                    acc = CT<C>::mk(acc.x * s, acc.y * s);
                } else {
                    acc = cadd(cmul(wpx, xp), cmul(wmx, xm));
                    acc = cadd(acc, cadd(cmul(wpy[rr], yp), cmul(wmy[rr], ym)));
                    acc = cadd(acc, cadd(cmul(czp, pp), cmul(czm, pm)));
                }
                const C wcs = cadd(cadd(wcx, wcy[rr]), czc);
                const R kp = reinterpret_cast<const float *>(bc + OK)[tidx];
                const C diag = CT<C>::mk(kp * sc.zfac.x - sc.mu - wcs.x, kp * sc.zfac.y - wcs.y);
                acc = cadd(acc, cmul(diag, pc));
                C out = cmul(sc.sigma, acc);
                if (HAS_Y) out = cadd(out, sm_ld<S>(reinterpret_cast<const S *>(bc + OY), tidx));
                if (HAS_V) out = cadd(out, cmul(sc.gamma, sm_ld<S>(reinterpret_cast<const S *>(bc + OV), tidx)));
                out = cmul(sc.rho, out);
                St<S>::st(outp, g.s1 * 8 * rr, out);
            }
        }
        __syncthreads();                      // stage of plane pi - 1 is free
        if (tid == 0 && issued < nplanes) {
            issue(issued++, is_stage);        // is_stage == sm_ here
            if (++is_stage == kStages) is_stage = 0;
        }
        sm_ = sc_;
        sc_ = sp_;
        if (++sp_ == kStages) sp_ = 0;
        czp = czp_n;
        czm = czm_n;
        czc = czc_n;
    }
    // loads issued but never waited for (only after a timeout): wait, bounded
    if (tid == 0) {
        for (; waited + 1 < issued; ++waited) {
            if (!mbar_wait(&bar[w_stage], (unsigned)w_par)) break;
            if (++w_stage == kStages) { w_stage = 0; w_par ^= 1; }
        }
    }
}

// ---------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

// 3D map of a grid-shaped array of 4-byte elements (e per value), box bx x by x 1
static bool encode3(CUtensorMap *m, const void *base, const Geom &g, int e, int bx, int by)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[0] * e, (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * e * 4, (cuuint64_t)g.n[0] * g.n[1] * e * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Tma3Maps {
    CUtensorMap p[4], y[4], k;
    bool ok = false;
};

template <typename S>
Tma3Maps *tma3_create(const Geom &g, void *const *bufs, const float *kappa)
{
    if (g.dim != 3 || g.n[0] % 4 != 0) return nullptr;
    if ((reinterpret_cast<uintptr_t>(kappa) & 15) != 0) return nullptr;
    for (int b = 0; b < 4; ++b)
        if ((reinterpret_cast<uintptr_t>(bufs[b]) & 15) != 0) return nullptr;
    constexpr int E = TmaElt<S>::E, HL = TmaElt<S>::HL;
    Tma3Maps *t = new Tma3Maps();
    bool ok = true;
    for (int b = 0; b < 4 && ok; ++b) {
        ok = encode3(&t->p[b], bufs[b], g, E, E * (kTX + 2 * HL), kTY + 2) &&
             encode3(&t->y[b], bufs[b], g, E, E * kTX, kTY);
    }
    ok = ok && encode3(&t->k, kappa, g, 1, kTX, kTY);
    if (!ok) {
        delete t;
        return nullptr;
    }
    t->ok = true;
    return t;
}

void tma3_destroy(Tma3Maps *t) { delete t; }

template <typename S, bool HAS_Y, bool HAS_V>
static cudaError_t launch3t(const Geom &g, const typename St<S>::C *coef, const StepScalars<typename St<S>::C> &sc,
                            const Tma3Maps &t, int ip, int iy, int iv, S *pout, unsigned *err, cudaStream_t st)
{
    constexpr int SB = Tma3Geo<S>::stage_bytes(HAS_Y, HAS_V);
    constexpr size_t smem = (size_t)SB * kStages + 128;
    static std::atomic<bool> configured[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev].load()) {
        cudaFuncSetAttribute(k_step3z_tma<S, HAS_Y, HAS_V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured[dev].store(true);
    }
    // segment length: about four waves of blocks
    const int64_t bxy = (int64_t)((g.n[0] + kTX - 1) / kTX) * ((g.n[1] + kTY - 1) / kTY);
    int64_t nseg = ((int64_t)sm_count() * 4 * 4 + bxy - 1) / bxy;
    if (nseg < 1) nseg = 1;
    int lz = (int)((g.n[2] + nseg - 1) / nseg);
    if (lz < 8) lz = 8;
    dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY, (g.n[2] + lz - 1) / lz);
    count_launch();
    k_step3z_tma<S, HAS_Y, HAS_V><<<grid, dim3(kTX, 8), smem, st>>>(g, coef, sc, t.p[ip], t.y[iy], t.k,
                                                                      t.y[iv < 0 ? 0 : iv], pout, lz, err);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_step3z_tma(const Geom &g, const typename St<S>::C *coef, const StepScalars<typename St<S>::C> &sc,
                              const Tma3Maps *t, int ip, int iy, int iv, S *pout, unsigned *err, cudaStream_t st)
{
    if (!t || !t->ok || ip < 0 || ip > 3 || iy > 3 || iv > 3) return cudaErrorInvalidValue;
    if (iy >= 0 && iv >= 0) return launch3t<S, true, true>(g, coef, sc, *t, ip, iy, iv, pout, err, st);
    if (iy >= 0) return launch3t<S, true, false>(g, coef, sc, *t, ip, iy, iv, pout, err, st);
    if (iv >= 0) return launch3t<S, false, true>(g, coef, sc, *t, ip, 0, iv, pout, err, st);
    return launch3t<S, false, false>(g, coef, sc, *t, ip, 0, iv, pout, err, st);
}

#define MXP_TINST(S)                                                                                     \
    template Tma3Maps *tma3_create<S>(const Geom &, void *const *, const float *);                      \
    template cudaError_t launch_step3z_tma<S>(const Geom &, const typename St<S>::C *,                  \
                                              const StepScalars<typename St<S>::C> &, const Tma3Maps *, \
                                              int, int, int, S *, unsigned *, cudaStream_t);
MXP_TINST(float2)
MXP_TINST(__nv_bfloat162)
#undef MXP_TINST

}  // namespace mxp
