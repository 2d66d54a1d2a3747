// Persistent 2D exp action: one cooperative launch computes a whole
// exp(i t A_s) v action (all S sub-steps x m Taylor-Horner steps, Def. psi).
//
// Each CTA owns one tile of the grid for the whole action.  The tile plus a
// K-cell ring lives in shared memory (two ping-pong buffers); y (the sub-step
// start vector) stays in registers.  One pass = K Horner steps on the region;
// afterwards the tile interior is exact, the CTA publishes the K-wide strips
// along its tile edges to a global exchange buffer and posts its pass number
// (epoch), waits until its eight neighbours have posted theirs (point-to-point,
// no grid-wide barrier), and refreshes its ring from their strips.  Global
// traffic per pass is only these strips (L2-resident), and there is one launch
// per action instead of one per pass.
//
// Every wait polls a bounded number of times; on timeout it sets an error word
// and every CTA leaves the pass loop, so the kernel always ends.
// Co-residency of all CTAs is guaranteed by the cooperative launch (the launch
// fails instead of deadlocking when the grid does not fit).
#include <algorithm>

#include "mxp_internal.h"

namespace mxp {

struct PersistArgs {
    int n0, n1, nmax, npml;
    int txo, tyo, ntx, nty;      // tile extents and tile counts
    const float2 *coef;          // coefficient table scaled by h^2 (operator in dimensionless units)
    const float *kappa;
    float2 zfac;                 // 1 + i s
    float h2;                    // h^2: scales kappa (1 + i s)
    const float *tau;            // per step: tau / h^2 (operator scaled by h^2), npass * K
    int npass, pass_per_sub;     // passes in total and per sub-step
    float2 rho;                  // e^{i t mu}: multiplies the result (undoes the shift)
    unsigned *bar;               // [0] arrival count, [1] generation, [2] error flag, [4..] tile epochs
    // psi_1 by sub-steps (nullptr for exp): after sub-step j (1-based) the tile
    // gains wcoef[j-1] * w (w in the storage type S)
    const void *w;
    const float2 *wcoef;
    // ghost-point faces x-, x+, y-, y+ (nullptr = zero Dirichlet): diagonal term
    // of each boundary cell, scaled by h^2, indexed by the position along the face
    const float2 *face[4];
    int nfaces;
};

constexpr long long kBarrierSpinLimit = 1ll << 24;   // x >= 32 ns sleep: about a second
constexpr long long kNeighbourPollLimit = 1ll << 21;  // L2 polls (~0.5 us each): about a second

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks,
                                             long long limit = kBarrierSpinLimit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile unsigned *verr = bar + 2;
        int ok = 1;
        __threadfence();
        const unsigned gen = *vgen;
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*vgen == gen) {
                if (++it > limit || *verr != 0u) {
                    atomicExch(bar + 2, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok && (*verr == 0u);
    }
    __syncthreads();
    return s_ok != 0;
}

// Point-to-point pass synchronisation: after publishing its strips for pass p a
// CTA posts epoch p + 1, then waits until each of its (up to eight) neighbour
// tiles has posted at least p + 1.  A CTA is therefore at most one pass ahead of
// any neighbour, which keeps the two exchange buffers safe.  Lanes 0..8 of warp
// 0 poll one neighbour each (lane 4 is the tile itself), so the wait costs one
// L2 round trip when the neighbours are already there.  Bounded polling: on
// timeout the error word is set and the caller stops.
// The epoch word is written with release semantics after the CTA barrier (so
// the strips every thread of the CTA stored before it are visible first) and
// read with acquire semantics before the closing CTA barrier (so the ring loads
// that follow it see the neighbours' strips): the ordering of a fence on each
// side without a full fence.
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// entry_barrier = false when the caller has just passed a CTA barrier after its
// last store of the strips (nothing to order again).
__device__ __forceinline__ bool neighbour_sync(unsigned *bar, int bx, int by, int ntx, int nty,
                                               unsigned epoch, bool entry_barrier = true)
{
    __shared__ int s_ok2;
    if (entry_barrier) __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned *flags = bar + 4;
        volatile unsigned *verr = bar + 2;
        if (lane == 0) st_release_gpu(bar + 4 + (by * ntx + bx) * kPersistFlagStride, epoch);
        int ok = 1;
        if (lane < 9 && lane != 4) {
            const int nx = bx + lane % 3 - 1, ny = by + lane / 3 - 1;
            if (nx >= 0 && ny >= 0 && nx < ntx && ny < nty) {
                long long it = 0;
                while (ld_acquire_gpu(flags + (ny * ntx + nx) * kPersistFlagStride) < epoch) {
                    if (++it > kNeighbourPollLimit || *verr != 0u) {
                        atomicExch(bar + 2, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) s_ok2 = ok && (*verr == 0u);
    }
    __syncthreads();
    return s_ok2 != 0;
}

template <typename S, int K, int BX, int BG, int R, int CH>
__global__ void __launch_bounds__(BX *BG, 1) k_persist2d(PersistArgs a, const S *__restrict__ x,
                                                         S *__restrict__ ex0,
                                                         S *__restrict__ ex1,
                                                         S *__restrict__ out)
{
    static_assert(K % 2 == 0, "K must be even: each pass starts and ends in buffer 0");
    static_assert(R % CH == 0, "rows per thread must be a multiple of the chunk");
    constexpr int PX = BX + 2;
    constexpr int PY = BG * R + 2;
    extern __shared__ float2 sm[];
    float2 *b0 = sm;
    float2 *b1 = sm + PY * PX;
    float2 *cy = b1 + PY * PX;          // [BG*R][3] y-axis coefficients wp, wm, wc of region rows
    float *ks = reinterpret_cast<float *>(cy + 3 * BG * R);   // [BG*R][BX] kappa of the region

    const int tx = threadIdx.x % BX;
    const int grp = threadIdx.x / BX;
    const int bx = blockIdx.x % a.ntx, by = blockIdx.x / a.ntx;
    const int RW = a.txo + 2 * K, RH = a.tyo + 2 * K;       // region extents
    const int gx0 = bx * a.txo - K, gy0 = by * a.tyo - K;
    const int gx = gx0 + tx;
    const bool colok = (tx < RW);
    const bool inx = colok && gx >= 0 && gx < a.n0;
    const int n0 = a.n0, n1 = a.n1, nm = a.nmax;
    const float h2 = a.h2;

    for (int i = threadIdx.x; i < 2 * PY * PX; i += BX * BG) sm[i] = make_float2(0.f, 0.f);
    for (int r = threadIdx.x; r < BG * R; r += BX * BG) {
        const int gy = gy0 + r;
        float2 wp = make_float2(0.f, 0.f), wm = make_float2(0.f, 0.f), wc = make_float2(0.f, 0.f);
        if (gy >= 0 && gy < n1) {
            wp = a.coef[3 * nm + gy];
            wm = a.coef[4 * nm + gy];
            wc = a.coef[5 * nm + gy];
        }
        cy[3 * r] = wp;
        cy[3 * r + 1] = wm;
        cy[3 * r + 2] = wc;
    }
    float2 wpx = make_float2(0.f, 0.f), wmx = make_float2(0.f, 0.f), wcx = make_float2(0.f, 0.f);
    if (inx) {
        wpx = a.coef[gx];
        wmx = a.coef[nm + gx];
        wcx = a.coef[2 * nm + gx];
    }
    const float2 zh = make_float2(a.zfac.x * h2, a.zfac.y * h2);
    __syncthreads();

    // per-point state: y (sub-step start) in registers, kappa in shared memory
    float2 yr[R];
    unsigned inmask = 0u;     // point inside the grid and the region
    unsigned tilemask = 0u;   // point inside this CTA's tile
    unsigned stripmask = 0u;  // tile point within K of the tile edge (published)
    unsigned facemask = 0u;   // point on a sound-hard or absorbing face of the grid
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ry = grp * R + r;
        const int gy = gy0 + ry;
        const bool in = inx && ry < RH && gy >= 0 && gy < n1;
        if (in && a.nfaces &&
            ((a.face[0] && gx == 0) || (a.face[1] && gx == n0 - 1) || (a.face[2] && gy == 0) ||
             (a.face[3] && gy == n1 - 1)))
            facemask |= 1u << r;
        const int64_t q = in ? (int64_t)gy * n0 + gx : 0;
        const float2 p0 = St<S>::ld(x, q);
        ks[ry * BX + tx] = a.kappa[q];
        yr[r] = in ? p0 : make_float2(0.f, 0.f);
        if (in) {
            inmask |= 1u << r;
            b0[(ry + 1) * PX + tx + 1] = p0;
            const bool intile = tx >= K && tx < K + a.txo && ry >= K && ry < K + a.tyo;
            if (intile) {
                tilemask |= 1u << r;
                if (tx < 2 * K || tx >= a.txo || ry < 2 * K || ry >= a.tyo) stripmask |= 1u << r;
            }
        }
    }
    __syncthreads();

    bool alive = true;
    for (int pass = 0; pass < a.npass && alive; ++pass) {
#pragma unroll 1
        for (int s = 0; s < K; ++s) {
            const float2 *src = (s & 1) ? b1 : b0;
            float2 *dst = (s & 1) ? b0 : b1;
            const float tau = a.tau[pass * K + s];
            const int r0 = grp * R;
            float2 up = src[r0 * PX + tx + 1];
            float2 cen = src[(r0 + 1) * PX + tx + 1];
            // rows in chunks of CH: all shared loads of a chunk are issued before
            // any of its stores, so they overlap instead of waiting row by row
#pragma unroll
            for (int c = 0; c < R; c += CH) {
                if (r0 + c >= RH) break;                 // uniform across the warp
                float2 dn[CH], e[CH], w[CH], o[CH];
                float kk[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int ry = r0 + c + j;
                    dn[j] = src[(ry + 2) * PX + tx + 1];
                    e[j] = src[(ry + 1) * PX + tx + 2];
                    w[j] = src[(ry + 1) * PX + tx];
                    kk[j] = ks[ry * BX + tx];
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int ry = r0 + c + j;
                    const float2 wpy = cy[3 * ry], wmy = cy[3 * ry + 1], wcy = cy[3 * ry + 2];
                    // scaled diagonal h^2 (kappa (1 + i s) - wc_x - wc_y); mu is folded in wc
                    const float dx = fmaf(kk[j], zh.x, -(wcx.x + wcy.x));
                    const float dy = fmaf(kk[j], zh.y, -(wcx.y + wcy.y));
                    // q = wpx e + wmx w + wpy dn + wmy up + d cen as one FMA chain per component
                    const float2 e_ = e[j], w_ = w[j], n_ = dn[j];
                    float qx = wpx.x * e_.x;
                    qx = fmaf(-wpx.y, e_.y, qx);
                    qx = fmaf(wmx.x, w_.x, qx);
                    qx = fmaf(-wmx.y, w_.y, qx);
                    qx = fmaf(wpy.x, n_.x, qx);
                    qx = fmaf(-wpy.y, n_.y, qx);
                    qx = fmaf(wmy.x, up.x, qx);
                    qx = fmaf(-wmy.y, up.y, qx);
                    qx = fmaf(dx, cen.x, qx);
                    qx = fmaf(-dy, cen.y, qx);
                    float qy = wpx.x * e_.y;
                    qy = fmaf(wpx.y, e_.x, qy);
                    qy = fmaf(wmx.x, w_.y, qy);
                    qy = fmaf(wmx.y, w_.x, qy);
                    qy = fmaf(wpy.x, n_.y, qy);
                    qy = fmaf(wpy.y, n_.x, qy);
                    qy = fmaf(wmy.x, up.y, qy);
                    qy = fmaf(wmy.y, up.x, qy);
                    qy = fmaf(dx, cen.y, qy);
                    qy = fmaf(dy, cen.x, qy);
                    o[j] = make_float2(fmaf(-tau, qy, yr[c + j].x), fmaf(tau, qx, yr[c + j].y));
                    up = cen;
                    cen = dn[j];
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int ry = r0 + c + j;
                    if ((inmask >> (c + j)) & 1u) dst[(ry + 1) * PX + tx + 1] = o[j];
                }
            }
            if (facemask) {
                // boundary rows of a ghost-point face: the ghost is a multiple of the
                // row's own unknown, so q gains face * p (added to this thread's cells)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((facemask >> r) & 1u) {
                        const int ry = r0 + r, gy = gy0 + ry;
                        float2 f = make_float2(0.f, 0.f);
                        if (a.face[0] && gx == 0) f = cadd(f, a.face[0][gy]);
                        if (a.face[1] && gx == n0 - 1) f = cadd(f, a.face[1][gy]);
                        if (a.face[2] && gy == 0) f = cadd(f, a.face[2][gx]);
                        if (a.face[3] && gy == n1 - 1) f = cadd(f, a.face[3][gx]);
                        const float2 fp = cmul(f, src[(ry + 1) * PX + tx + 1]);
                        float2 &cell = dst[(ry + 1) * PX + tx + 1];
                        cell = make_float2(fmaf(-tau, fp.y, cell.x), fmaf(tau, fp.x, cell.y));
                    }
                }
            }
            __syncthreads();
        }
        if (a.w && ((pass + 1) % a.pass_per_sub) == 0) {
            // u_{j+1} = exp(h M') u_j + c_j w on the tile's own cells; the ring gets
            // the same from the neighbours' strips
            const float2 cj = a.wcoef[(pass + 1) / a.pass_per_sub - 1];
            const S *w = static_cast<const S *>(a.w);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if ((tilemask >> r) & 1u) {
                    const int ry = grp * R + r;
                    float2 &cell = b0[(ry + 1) * PX + tx + 1];
                    cell = cadd(cell, cmul(cj, St<S>::ld(w, (int64_t)(gy0 + ry) * n0 + gx)));
                }
            }
        }
        if (pass == a.npass - 1) break;
        // publish the tile's edge strips, meet, pull the ring from the neighbours
        S *ex = (pass & 1) ? ex1 : ex0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((stripmask >> r) & 1u) {
                const int ry = grp * R + r;
                const int64_t q = (int64_t)(gy0 + ry) * n0 + gx;
                St<S>::st(ex, q, b0[(ry + 1) * PX + tx + 1]);
            }
        }
        alive = neighbour_sync(a.bar, bx, by, a.ntx, a.nty, (unsigned)(pass + 1));
        if (!alive) break;
        const bool sub_end = ((pass + 1) % a.pass_per_sub) == 0;
        // ring refresh: issue every L2 load first (clamped addresses), then store
        const unsigned ring = inmask & ~tilemask;
        if (ring) {
            float2 rv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ry = grp * R + r;
                const int64_t q = ((ring >> r) & 1u) ? (int64_t)(gy0 + ry) * n0 + gx : 0;
                if (sizeof(S) == 8) {
                    rv[r] = __ldcg(reinterpret_cast<const float2 *>(ex) + q);
                } else {
                    const unsigned u = __ldcg(reinterpret_cast<const unsigned *>(ex) + q);
                    rv[r] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if ((ring >> r) & 1u) b0[(grp * R + r + 1) * PX + tx + 1] = rv[r];
        }
        __syncthreads();
        if (sub_end) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if ((inmask >> r) & 1u) yr[r] = b0[(grp * R + r + 1) * PX + tx + 1];
        }
    }
    if (alive) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((tilemask >> r) & 1u) {
                const int ry = grp * R + r;
                St<S>::st(out, (int64_t)(gy0 + ry) * n0 + gx, cmul(a.rho, b0[(ry + 1) * PX + tx + 1]));
            }
        }
    }
}

// One Taylor-Horner step over a thread's R rows of its two columns (the body of
// k_persist2d_x2): all shared loads of a chunk of CH rows are issued before its
// arithmetic, then the chunk's results are stored.
// Shared-memory index of the thread's column l (0: its first, 1: its second
// column) in region row ry.  Interleaved rows hold the cells in order,
// (ry + 1) PX + cx + 2; split rows hold all first columns of the column pairs,
// then all second columns, each half with one zero cell on both sides, so that
// the west neighbour (the second column of the thread to the left) and the east
// neighbour (the first column of the thread to the right) are contiguous over
// the lanes of a warp: two shared-memory wavefronts per load instead of four.
template <bool SPLIT, int PX, int BXH>
__device__ __forceinline__ int x2_cell(int ry, int tx, int l)
{
    return SPLIT ? (ry + 1) * PX + (l ? BXH + 3 : 1) + tx : (ry + 1) * PX + 2 * tx + l + 2;
}

template <int R, int CH, int PX, int BXH, bool SPLIT>
__device__ __forceinline__ void x2_step_rows(const float2 *__restrict__ src, float2 *__restrict__ dst,
                                             const float2 *__restrict__ cy, const float2 *__restrict__ ks,
                                             int r0, int RH, int cx0, int tx, const float2 (&wpx)[2],
                                             const float2 (&wmx)[2], const float2 (&wcx)[2], float2 zh,
                                             float tau, const float2 (&y0r)[R], const float2 (&y1r)[R])
{
    auto ld_pair = [&](int ry) -> float4 {     // both columns of region row ry
        if (SPLIT) {
            const float2 lo = src[x2_cell<true, PX, BXH>(ry, tx, 0)], hi = src[x2_cell<true, PX, BXH>(ry, tx, 1)];
            return make_float4(lo.x, lo.y, hi.x, hi.y);
        }
        return *reinterpret_cast<const float4 *>(src + (ry + 1) * PX + cx0 + 2);
    };
    float4 up = ld_pair(r0 - 1);
    float4 cen = ld_pair(r0);
#pragma unroll
    for (int c = 0; c < R; c += CH) {
        if (r0 + c >= RH) break;                 // uniform across the row group
        float4 dn[CH];
        float2 wl[CH], er[CH], kk[CH];
        float4 o[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int ry = r0 + c + j;
            dn[j] = ld_pair(ry + 1);
            if (SPLIT) {
                wl[j] = src[x2_cell<true, PX, BXH>(ry, tx, 1) - 1];
                er[j] = src[x2_cell<true, PX, BXH>(ry, tx, 0) + 1];
            } else {
                wl[j] = src[(ry + 1) * PX + cx0 + 1];
                er[j] = src[(ry + 1) * PX + cx0 + 4];
            }
            kk[j] = ks[ry * BXH + tx];
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int ry = r0 + c + j;
            const float2 wpy = cy[3 * ry], wmy = cy[3 * ry + 1], wcy = cy[3 * ry + 2];
            const float2 cA = make_float2(cen.x, cen.y), cB = make_float2(cen.z, cen.w);
            const float2 uA = make_float2(up.x, up.y), uB = make_float2(up.z, up.w);
            const float2 nA = make_float2(dn[j].x, dn[j].y), nB = make_float2(dn[j].z, dn[j].w);
            float2 res[2];
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const float2 e_ = l ? er[j] : cB, w_ = l ? cA : wl[j];
                const float2 n_ = l ? nB : nA, u_ = l ? uB : uA, c_ = l ? cB : cA;
                const float kv = l ? kk[j].y : kk[j].x;
                const float dx = fmaf(kv, zh.x, -(wcx[l].x + wcy.x));
                const float dy = fmaf(kv, zh.y, -(wcx[l].y + wcy.y));
                // q = wpx e + wmx w + wpy n + wmy u + d c as one FMA chain per component
                float qx = wpx[l].x * e_.x;
                qx = fmaf(-wpx[l].y, e_.y, qx);
                qx = fmaf(wmx[l].x, w_.x, qx);
                qx = fmaf(-wmx[l].y, w_.y, qx);
                qx = fmaf(wpy.x, n_.x, qx);
                qx = fmaf(-wpy.y, n_.y, qx);
                qx = fmaf(wmy.x, u_.x, qx);
                qx = fmaf(-wmy.y, u_.y, qx);
                float qy = wpx[l].x * e_.y;
                qy = fmaf(wpx[l].y, e_.x, qy);
                qy = fmaf(wmx[l].x, w_.y, qy);
                qy = fmaf(wmx[l].y, w_.x, qy);
                qy = fmaf(wpy.x, n_.y, qy);
                qy = fmaf(wpy.y, n_.x, qy);
                qy = fmaf(wmy.x, u_.y, qy);
                qy = fmaf(wmy.y, u_.x, qy);
                qx = fmaf(dx, c_.x, qx);
                qx = fmaf(-dy, c_.y, qx);
                qy = fmaf(dx, c_.y, qy);
                qy = fmaf(dy, c_.x, qy);
                const float2 yv = l ? y1r[c + j] : y0r[c + j];
                res[l] = make_float2(fmaf(-tau, qy, yv.x), fmaf(tau, qx, yv.y));
            }
            o[j] = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
            up = cen;
            cen = dn[j];
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            if (SPLIT) {
                dst[x2_cell<true, PX, BXH>(r0 + c + j, tx, 0)] = make_float2(o[j].x, o[j].y);
                dst[x2_cell<true, PX, BXH>(r0 + c + j, tx, 1)] = make_float2(o[j].z, o[j].w);
            } else {
                *reinterpret_cast<float4 *>(dst + (r0 + c + j + 1) * PX + cx0 + 2) = o[j];
            }
        }
    }
}

// The same exp / psi_1 action with two adjacent columns per thread.  The east
// neighbour of the first column and the west neighbour of the second are the
// other column's centre (registers), the row below comes as one 16-byte load
// for both, and kappa of both as one 8-byte load: about half the shared loads
// per point of k_persist2d.  Cells outside the grid start at zero, have y = 0
// and meet only zero coefficients, so they stay exactly zero and every row pair
// is stored unmasked; cells past the region's edge only spread garbage inward
// by one cell per step, which the K-cell ring absorbs.  FACES = true adds the
// ghost-point face terms as k_persist2d does (a separate instantiation, so the
// face-free kernel keeps its register allocation).
template <typename S, int K, int BXH, int BG, int R, int CH, bool FACES, bool SPLIT>
__global__ void __launch_bounds__(BXH *BG, 1) k_persist2d_x2(PersistArgs a, const S *__restrict__ x,
                                                             S *__restrict__ ex0,
                                                             S *__restrict__ ex1,
                                                             S *__restrict__ out)
{
    static_assert(K % 2 == 0, "K must be even: each pass starts and ends in buffer 0");
    static_assert(R % CH == 0, "rows per thread must be a multiple of the chunk");
    constexpr int BX = 2 * BXH;                 // region columns
    constexpr int PX = BX + 4;                  // padded row: cell (ry, cx) at (ry + 1) PX + cx + 2
    constexpr int PY = BG * R + 2;
    extern __shared__ __align__(16) float2 sm[];
    float2 *b0 = sm;
    float2 *b1 = sm + PY * PX;
    float2 *cy = b1 + PY * PX;                  // [BG*R][3] y-axis coefficients wp, wm, wc
    float2 *ks = cy + 3 * BG * R;               // [BG*R][BXH] kappa of the column pair

    const int tx = threadIdx.x % BXH;
    const int grp = threadIdx.x / BXH;
    const int bx = blockIdx.x % a.ntx, by = blockIdx.x / a.ntx;
    const int RW = a.txo + 2 * K, RH = a.tyo + 2 * K;
    const int gx0 = bx * a.txo - K, gy0 = by * a.tyo - K;
    const int cx0 = 2 * tx;                     // region column of the first cell
    const int n0 = a.n0, n1 = a.n1, nm = a.nmax;
    const float h2 = a.h2;
    int gx[2];
    bool inx[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        gx[l] = gx0 + cx0 + l;
        inx[l] = cx0 + l < RW && gx[l] >= 0 && gx[l] < n0;
    }

    for (int i = threadIdx.x; i < 2 * PY * PX; i += BXH * BG) sm[i] = make_float2(0.f, 0.f);
    for (int r = threadIdx.x; r < BG * R; r += BXH * BG) {
        const int gy = gy0 + r;
        float2 wp = make_float2(0.f, 0.f), wm = make_float2(0.f, 0.f), wc = make_float2(0.f, 0.f);
        if (gy >= 0 && gy < n1) {
            wp = a.coef[3 * nm + gy];
            wm = a.coef[4 * nm + gy];
            wc = a.coef[5 * nm + gy];
        }
        cy[3 * r] = wp;
        cy[3 * r + 1] = wm;
        cy[3 * r + 2] = wc;
    }
    float2 wpx[2], wmx[2], wcx[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        wpx[l] = wmx[l] = wcx[l] = make_float2(0.f, 0.f);
        if (inx[l]) {
            wpx[l] = a.coef[gx[l]];
            wmx[l] = a.coef[nm + gx[l]];
            wcx[l] = a.coef[2 * nm + gx[l]];
        }
    }
    const float2 zh = make_float2(a.zfac.x * h2, a.zfac.y * h2);
    __syncthreads();

    float2 y0r[R], y1r[R];
    unsigned inmask[2] = {0u, 0u}, tilemask[2] = {0u, 0u}, stripmask[2] = {0u, 0u};
    unsigned facemask[2] = {0u, 0u};
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ry = grp * R + r;
        const int gy = gy0 + ry;
        float kap[2];
        float2 pv[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool in = inx[l] && ry < RH && gy >= 0 && gy < n1;
            const int64_t q = in ? (int64_t)gy * n0 + gx[l] : 0;
            pv[l] = in ? St<S>::ld(x, q) : make_float2(0.f, 0.f);
            kap[l] = a.kappa[q];
            if (FACES && in && a.nfaces &&
                ((a.face[0] && gx[l] == 0) || (a.face[1] && gx[l] == n0 - 1) || (a.face[2] && gy == 0) ||
                 (a.face[3] && gy == n1 - 1)))
                facemask[l] |= 1u << r;
            if (in) {
                inmask[l] |= 1u << r;
                b0[x2_cell<SPLIT, PX, BXH>(ry, tx, l)] = pv[l];
                const int cx = cx0 + l;
                const bool intile = cx >= K && cx < K + a.txo && ry >= K && ry < K + a.tyo;
                if (intile) {
                    tilemask[l] |= 1u << r;
                    if (cx < 2 * K || cx >= a.txo || ry < 2 * K || ry >= a.tyo) stripmask[l] |= 1u << r;
                }
            }
        }
        ks[ry * BXH + tx] = make_float2(kap[0], kap[1]);
        y0r[r] = pv[0];
        y1r[r] = pv[1];
    }
    __syncthreads();
    bool alive = true;
    for (int pass = 0; pass < a.npass && alive; ++pass) {
        const bool early_pub = pass < a.npass - 1 && !(a.w && ((pass + 1) % a.pass_per_sub) == 0);
#pragma unroll 1
        for (int s = 0; s < K; ++s) {
            const float2 *src = (s & 1) ? b1 : b0;
            float2 *dst = (s & 1) ? b0 : b1;
            const float tau = a.tau[pass * K + s];
            const int r0 = grp * R;
            x2_step_rows<R, CH, PX, BXH, SPLIT>(src, dst, cy, ks, r0, RH, cx0, tx, wpx, wmx, wcx, zh, tau, y0r, y1r);
            if (FACES && (facemask[0] | facemask[1])) {
                // boundary rows of a ghost-point face: q gains face * p on those cells
#pragma unroll
                for (int l = 0; l < 2; ++l) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if ((facemask[l] >> r) & 1u) {
                            const int ry = r0 + r, gy = gy0 + ry, gxl = gx[l];
                            float2 f = make_float2(0.f, 0.f);
                            if (a.face[0] && gxl == 0) f = cadd(f, a.face[0][gy]);
                            if (a.face[1] && gxl == n0 - 1) f = cadd(f, a.face[1][gy]);
                            if (a.face[2] && gy == 0) f = cadd(f, a.face[2][gxl]);
                            if (a.face[3] && gy == n1 - 1) f = cadd(f, a.face[3][gxl]);
                            const int ci = x2_cell<SPLIT, PX, BXH>(ry, tx, l);
                            const float2 fp = cmul(f, src[ci]);
                            dst[ci] = make_float2(fmaf(-tau, fp.y, dst[ci].x), fmaf(tau, fp.x, dst[ci].y));
                        }
                    }
                }
            }
            if (s == K - 1 && early_pub) {
                // publish the strips from this thread's own new cells (written by it
                // above) before the step's barrier, so the global stores are in flight
                S *ex = (pass & 1) ? ex1 : ex0;
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    const int ry = r0 + r;
#pragma unroll
                    for (int l = 0; l < 2; ++l)
                        if ((stripmask[l] >> r) & 1u)
                            St<S>::st(ex, (int64_t)(gy0 + ry) * n0 + gx[l], dst[x2_cell<SPLIT, PX, BXH>(ry, tx, l)]);
                }
            }
            __syncthreads();
        }
        if (a.w && ((pass + 1) % a.pass_per_sub) == 0) {
            const float2 cj = a.wcoef[(pass + 1) / a.pass_per_sub - 1];
            const S *w = static_cast<const S *>(a.w);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ry = grp * R + r;
#pragma unroll
                for (int l = 0; l < 2; ++l)
                    if ((tilemask[l] >> r) & 1u) {
                        float2 &cell = b0[x2_cell<SPLIT, PX, BXH>(ry, tx, l)];
                        cell = cadd(cell, cmul(cj, St<S>::ld(w, (int64_t)(gy0 + ry) * n0 + gx[l])));
                    }
            }
        }
        if (pass == a.npass - 1) break;
        S *ex = (pass & 1) ? ex1 : ex0;
        if (!early_pub) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ry = grp * R + r;
#pragma unroll
                for (int l = 0; l < 2; ++l)
                    if ((stripmask[l] >> r) & 1u)
                        St<S>::st(ex, (int64_t)(gy0 + ry) * n0 + gx[l], b0[x2_cell<SPLIT, PX, BXH>(ry, tx, l)]);
            }
        }
        // after an early publish the last step's barrier already ordered the strips
        alive = neighbour_sync(a.bar, bx, by, a.ntx, a.nty, (unsigned)(pass + 1), !early_pub);
        if (!alive) break;
        const bool sub_end = ((pass + 1) % a.pass_per_sub) == 0;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const unsigned ring = inmask[l] & ~tilemask[l];
            if (ring) {
                float2 rv[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int ry = grp * R + r;
                    const int64_t q = ((ring >> r) & 1u) ? (int64_t)(gy0 + ry) * n0 + gx[l] : 0;
                    if (sizeof(S) == 8) {
                        rv[r] = __ldcg(reinterpret_cast<const float2 *>(ex) + q);
                    } else {
                        const unsigned u = __ldcg(reinterpret_cast<const unsigned *>(ex) + q);
                        rv[r] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((ring >> r) & 1u) b0[x2_cell<SPLIT, PX, BXH>(grp * R + r, tx, l)] = rv[r];
            }
        }
        __syncthreads();
        if (sub_end) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ry = grp * R + r;
                if ((inmask[0] >> r) & 1u) y0r[r] = b0[x2_cell<SPLIT, PX, BXH>(ry, tx, 0)];
                if ((inmask[1] >> r) & 1u) y1r[r] = b0[x2_cell<SPLIT, PX, BXH>(ry, tx, 1)];
            }
        }
    }
    if (alive) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int ry = grp * R + r;
#pragma unroll
            for (int l = 0; l < 2; ++l)
                if ((tilemask[l] >> r) & 1u)
                    St<S>::st(out, (int64_t)(gy0 + ry) * n0 + gx[l], cmul(a.rho, b0[x2_cell<SPLIT, PX, BXH>(ry, tx, l)]));
        }
    }
}

struct PCfg {
    int K, BX, BG, R;
    int x2;          // 1: two columns per thread (k_persist2d_x2, BX / 2 threads per row group)
    int faces;       // adds ghost-point face terms
};
// Configuration 9 is configuration 6 with the shared loads of 7 rows (instead of 2)
// issued ahead of their arithmetic (more loads in flight per thread, 160 registers);
// configuration 10 is 9 with split rows (x2_cell).
static const PCfg kPCfgs[] = {{2, 128, 4, 18, 0, 1}, {4, 96, 4, 28, 0, 1}, {4, 96, 8, 14, 0, 1},
                               {4, 96, 9, 12, 0, 1},  {2, 128, 8, 10, 0, 1}, {6, 96, 4, 28, 0, 1},
                               {6, 96, 8, 14, 1, 0},  {4, 96, 8, 14, 1, 0},  {6, 96, 8, 14, 1, 1},
                               {6, 96, 8, 14, 1, 0},  {6, 96, 8, 14, 1, 0}};
constexpr int kNumP = sizeof(kPCfgs) / sizeof(kPCfgs[0]);

int persist2d_num_cfgs() { return kNumP; }
int persist2d_cfg_k(int id) { return kPCfgs[id].K; }
bool persist2d_cfg_faces(int id) { return id >= 0 && id < kNumP && kPCfgs[id].faces; }
static int cfg_threads(const PCfg &c) { return c.x2 ? c.BX / 2 * c.BG : c.BX * c.BG; }

template <typename S, int K, int BX, int BG, int R>
static void *kernel_ptr() { return (void *)k_persist2d<S, K, BX, BG, R, (R % 4 == 0) ? 4 : 2>; }

template <int R>
constexpr int chunk_rows() { return (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 1; }

template <typename S, int K, int BX, int BG, int R, bool F, int CH = chunk_rows<R>(), bool SPLIT = false>
static void *kernel_ptr_x2() { return (void *)k_persist2d_x2<S, K, BX / 2, BG, R, CH, F, SPLIT>; }

template <typename S, int K, int BX, int BG, int R>
static size_t smem_bytes_x2()
{
    return (size_t)(2 * (BG * R + 2) * (BX + 4) + 3 * BG * R) * sizeof(float2) +
           (size_t)BG * R * BX * sizeof(float);
}

template <typename S, int K, int BX, int BG, int R>
static size_t smem_bytes()
{
    return (size_t)(2 * (BG * R + 2) * (BX + 2) + 3 * BG * R) * sizeof(float2) +
           (size_t)BG * R * BX * sizeof(float);
}

template <typename S>
static void cfg_info(int id, void **fn, size_t *smem)
{
    switch (id) {
    case 0: *fn = kernel_ptr<S, 2, 128, 4, 18>(); *smem = smem_bytes<S, 2, 128, 4, 18>(); break;
    case 1: *fn = kernel_ptr<S, 4, 96, 4, 28>(); *smem = smem_bytes<S, 4, 96, 4, 28>(); break;
    case 2: *fn = kernel_ptr<S, 4, 96, 8, 14>(); *smem = smem_bytes<S, 4, 96, 8, 14>(); break;
    case 3: *fn = kernel_ptr<S, 4, 96, 9, 12>(); *smem = smem_bytes<S, 4, 96, 9, 12>(); break;
    case 4: *fn = kernel_ptr<S, 2, 128, 8, 10>(); *smem = smem_bytes<S, 2, 128, 8, 10>(); break;
    case 5: *fn = kernel_ptr<S, 6, 96, 4, 28>(); *smem = smem_bytes<S, 6, 96, 4, 28>(); break;
    case 6: *fn = kernel_ptr_x2<S, 6, 96, 8, 14, false>(); *smem = smem_bytes_x2<S, 6, 96, 8, 14>(); break;
    case 7: *fn = kernel_ptr_x2<S, 4, 96, 8, 14, false>(); *smem = smem_bytes_x2<S, 4, 96, 8, 14>(); break;
    case 8: *fn = kernel_ptr_x2<S, 6, 96, 8, 14, true>(); *smem = smem_bytes_x2<S, 6, 96, 8, 14>(); break;
    case 9: *fn = kernel_ptr_x2<S, 6, 96, 8, 14, false, 7>(); *smem = smem_bytes_x2<S, 6, 96, 8, 14>(); break;
    default: *fn = kernel_ptr_x2<S, 6, 96, 8, 14, false, 7, true>(); *smem = smem_bytes_x2<S, 6, 96, 8, 14>(); break;
    }
}

// Tile plan: the largest number of tiles (at most `slots`, the co-resident
// CTAs) that minimises the region (tile plus K-cell ring) of one CTA, each tile
// no larger than txmax x tymax.  Every tile but the last one of a row or column
// is at least K cells wide on both axes, so the ring of a tile lies inside its
// eight neighbours: the point-to-point pass synchronisation only waits for
// those.  Returns false if no plan fits.
bool plan_tiles(int n0, int n1, int slots, int K, int txmax, int tymax, int *txo, int *tyo, int *ntx,
                int *nty)
{
    if (n0 < 1 || n1 < 1 || slots < 1 || K < 1 || txmax < 1 || tymax < 1) return false;
    const int ntx_min = (n0 + txmax - 1) / txmax, nty_min = (n1 + tymax - 1) / tymax;
    if ((long)ntx_min * nty_min > slots) return false;
    slots = std::min(slots, kPersistMaxTiles);   // per-tile epoch words available
    long best_area = -1;
    for (int tx_n = ntx_min; tx_n <= n0 && tx_n <= slots; ++tx_n) {
        const int a = (n0 + tx_n - 1) / tx_n;
        if (a < K && tx_n > ntx_min) break;       // narrower tiles would need a wider exchange
        const int ty_n_max = slots / tx_n;
        if (ty_n_max < nty_min) break;
        for (int ty_n = nty_min; ty_n <= ty_n_max && ty_n <= n1; ++ty_n) {
            const int b = (n1 + ty_n - 1) / ty_n;
            if (b < K && ty_n > nty_min) break;
            const long area = (long)(a + 2 * K) * (b + 2 * K);   // region per CTA
            if (best_area < 0 || area < best_area) {
                best_area = area;
                *txo = a;
                *tyo = b;
                *ntx = (n0 + a - 1) / a;
                *nty = (n1 + b - 1) / b;
            }
        }
    }
    return best_area > 0;
}

// Tile plan for configuration id on an n0 x n1 grid on this device.  Returns
// false if the grid does not fit on this device.
template <typename S>
bool persist2d_plan(int id, int n0, int n1, int device, int *txo, int *tyo, int *ntx, int *nty)
{
    if (id < 0 || id >= kNumP) return false;
    void *fn;
    size_t smem;
    cfg_info<S>(id, &fn, &smem);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int per_sm = 0, nsm = 0;
    const PCfg c = kPCfgs[id];
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, cfg_threads(c), smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    return plan_tiles(n0, n1, per_sm * nsm, c.K, c.BX - 2 * c.K, c.BG * c.R - 2 * c.K, txo, tyo, ntx, nty);
}

template <typename S>
cudaError_t launch_persist2d(int id, const Geom &g, int npml, const float2 *coef, const float *kappa,
                             float2 zfac, float h2, const float *tau_dev, int npass,
                             int pass_per_sub, float2 rho, unsigned *bar, int txo, int tyo,
                             int ntx, int nty, const S *x, S *ex0, S *ex1, S *out, cudaStream_t st,
                             const S *w, const float2 *wcoef, const float2 *const *faces)
{
    void *fn;
    size_t smem;
    cfg_info<S>(id, &fn, &smem);
    PersistArgs a;
    a.n0 = g.n[0];
    a.n1 = g.n[1];
    a.nmax = g.nmax;
    a.npml = npml;
    a.txo = txo;
    a.tyo = tyo;
    a.ntx = ntx;
    a.nty = nty;
    a.coef = coef;
    a.kappa = kappa;
    a.zfac = zfac;
    a.h2 = h2;
    a.tau = tau_dev;
    a.npass = npass;
    a.pass_per_sub = pass_per_sub;
    a.rho = rho;
    a.bar = bar;
    a.w = w;
    a.wcoef = wcoef;
    a.nfaces = 0;
    for (int f = 0; f < 4; ++f) {
        a.face[f] = faces ? faces[f] : nullptr;
        a.nfaces += (a.face[f] != nullptr);
    }
    void *args[] = {&a, (void *)&x, (void *)&ex0, (void *)&ex1, (void *)&out};
    const PCfg c = kPCfgs[id];
    // reset the arrival count, the generation and the tile epochs, but not the
    // error word bar[2]: a timeout of an earlier launch stays set until the host
    // reads it (and a launch that finds it set leaves its pass loop at once)
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(bar + 4, 0, (size_t)ntx * nty * kPersistFlagStride * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    count_launch();
    if (a.nfaces && !c.faces) return cudaErrorInvalidValue;   // this configuration has no face terms
    return cudaLaunchCooperativeKernel(fn, dim3(ntx * nty), dim3(cfg_threads(c)), args, smem, st);
}

// Self-test of the bounded grid barrier: the blocks wait for one more arrival
// than there are blocks, so every wait runs out after `limit` polls, sets the
// error word and returns.  Nothing here can wait forever.
__global__ void k_barrier_selftest(unsigned *bar, unsigned expected, long long limit)
{
    grid_barrier(bar, expected, limit);
}

cudaError_t barrier_selftest(unsigned *bar, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_barrier_selftest<<<2, 32, 0, st>>>(bar, 3u, 20000);
    return cudaGetLastError();
}

#define MXP_PINST(S)                                                                          \
    template bool persist2d_plan<S>(int, int, int, int, int *, int *, int *, int *);          \
    template cudaError_t launch_persist2d<S>(int, const Geom &, int, const float2 *, const float *, \
                                             float2, float, const float *, int, int, float2,  \
                                             unsigned *, int, int, int, int, const S *, S *,  \
                                             S *, S *, cudaStream_t, const S *, const float2 *, \
                                             const float2 *const *);
MXP_PINST(float2)
MXP_PINST(__nv_bfloat162)
#undef MXP_PINST

}  // namespace mxp

extern "C" int mxp_persist_tile_plan(int n0, int n1, int slots, int k, int txmax, int tymax, int *txo, int *tyo,
                                     int *ntx, int *nty)
{
    if (!txo || !tyo || !ntx || !nty) return 0;
    return mxp::plan_tiles(n0, n1, slots, k, txmax, tymax, txo, tyo, ntx, nty) ? 1 : 0;
}
