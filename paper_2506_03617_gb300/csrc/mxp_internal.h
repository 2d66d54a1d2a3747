// Internal declarations shared by the CUDA translation units of libmatexpre.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <atomic>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/matexpre.h"

namespace mxp {

// Record a message for mxp_last_error() (thread-local).
void note_error(const char *msg);

// Number of kernels this library has launched (process-wide).
extern std::atomic<long long> g_launch_count;
inline void count_launch(int n = 1) { g_launch_count.fetch_add(n, std::memory_order_relaxed); }

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

// ---------------------------------------------------------------- planning (plan.cu, host)
// Taylor plan of one exp / psi action: S sub-steps of a degree-m polynomial.
struct TaylorPlan {
    int S = 1;      // sub-steps
    int m = 1;      // Taylor degree per sub-step
    double nu = 0;  // norm bound used
};
// (S, m) minimising S*m with S (nu/S)^(m+1)/(m+1)! e^(nu/S) <= tol and
// nu/S <= theta_max; m rounded up to a multiple of kmult.
TaylorPlan make_plan(double nu, double tol, double theta_max, int kmult);
// Distinct coefficient classes of one axis: |wp| + |wm| and wc = wp + wm of
// every PML position plus one interior position.
struct AxisClasses {
    std::vector<double> off;
    std::vector<std::complex<double>> wc;
};
struct ShiftChoice {
    double mu = 0;   // real shift
    double nu = 0;   // row-sum bound of t (A_s - mu I) at that shift
};
// The shift mu minimising the row-sum bound of t (A_s - mu I) over the axis
// classes and omega^2/c^2 in [kmin, kmax] (golden-section search).
ShiftChoice choose_shift(const AxisClasses *cls, int dim, double kmin, double kmax, double shift_s,
                         double t);

// ---------------------------------------------------------------- complex math
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Storage traits: S is the type held in global memory for one complex value,
// C the complex type arithmetic happens in, R its real type.
template <typename S> struct St;
template <> struct St<double2> {
    using R = double; using C = double2;
    static __device__ __forceinline__ C ld(const double2 *p, int64_t i) { return p[i]; }
    static __device__ __forceinline__ void st(double2 *p, int64_t i, C v) { p[i] = v; }
    static __device__ __forceinline__ C from64(double2 v) { return v; }
};
template <> struct St<float2> {
    using R = float; using C = float2;
    static __device__ __forceinline__ C ld(const float2 *p, int64_t i) { return p[i]; }
    static __device__ __forceinline__ void st(float2 *p, int64_t i, C v) { p[i] = v; }
    static __device__ __forceinline__ C from64(double2 v) { return make_float2((float)v.x, (float)v.y); }
};
template <> struct St<__nv_bfloat162> {
    using R = float; using C = float2;
    static __device__ __forceinline__ C ld(const __nv_bfloat162 *p, int64_t i) { return __bfloat1622float2(p[i]); }
    static __device__ __forceinline__ void st(__nv_bfloat162 *p, int64_t i, C v) { p[i] = __float22bfloat162_rn(v); }
    static __device__ __forceinline__ C from64(double2 v) { return make_float2((float)v.x, (float)v.y); }
};

template <typename C> struct CT;
template <> struct CT<double2> { using R = double; static __host__ __device__ double2 mk(double a, double b) { return make_double2(a, b); } };
template <> struct CT<float2> { using R = float; static __host__ __device__ float2 mk(float a, float b) { return make_float2(a, b); } };

// ---------------------------------------------------------------- geometry
struct Geom {
    int dim;
    int n[3];          // unknowns per axis (1 for unused axes)
    int64_t s1, s2;    // strides of axes 1 and 2
    int64_t ntot;
    int nmax;          // max_d n[d]: row length of the coefficient table
    int fast = 0;      // 1: unknowns outside the PML use the real interior coefficient ih2
    int npml = 0;
    double ih2 = 0;    // 1 / h^2
};

// Scalars of one Taylor-Horner step  out = rho * (y + sigma * (A_s - mu) p + gamma * v)
template <typename C> struct StepScalars {
    C zfac;     // 1 + i s (or 1 for the unshifted operator)
    typename CT<C>::R mu;
    C sigma;
    C gamma;
    C rho;
    // ghost-point faces (x-, x+, y-, y+, z-, z+): diagonal term added on the
    // boundary rows of a sound-hard or absorbing face, indexed by the cell's
    // position on the face; nullptr = zero Dirichlet face.  nfaces = 0 skips all.
    const C *face[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int nfaces = 0;
};

// TMA-staged 3D sweep (tma3d.cu): tensor maps of the four 16-byte-per-unknown
// work buffers (as p with halo and as y / v tiles) and of kappa; nullptr when
// the grid does not qualify (3D with n0 a multiple of 4, 16-byte aligned
// buffers) or the driver offers no tensor-map encoder.
struct Tma3Maps;
template <typename S>
Tma3Maps *tma3_create(const Geom &g, void *const *bufs, const float *kappa);
void tma3_destroy(Tma3Maps *t);
// pout = one Taylor-Horner step as launch_step, reading p from buffer ip, y
// from buffer iy and v from buffer iv (-1 = none); err receives 1 on a wait
// timeout.
template <typename S>
cudaError_t launch_step3z_tma(const Geom &g, const typename St<S>::C *coef,
                              const StepScalars<typename St<S>::C> &sc, const Tma3Maps *t, int ip,
                              int iy, int iv, S *pout, unsigned *err, cudaStream_t st);

// ---------------------------------------------------------------- launchers
// coef: [dim][3][nmax] complex table: row 0 = a b+ / h^2, row 1 = a b- / h^2,
// row 2 = their sum (a = 1/s at the node, b+- = 1/s at the half nodes).
template <typename S>
void launch_step(const Geom &g, const typename St<S>::C *coef, const typename St<S>::R *kappa,
                 const StepScalars<typename St<S>::C> &sc, const S *pin, const S *y, const S *v,
                 S *pout, cudaStream_t st);

// Fused passes (2D): K consecutive Horner steps of one sub-step per launch,
// tiled through shared memory with a K-cell halo.  Step s uses
// sigma = i tau, gamma = (gamma_re, gamma_im) and, when rho_on, multiplies the
// result by rho.  cfg selects a tile shape (see fused2d.cu); returns false if
// the configuration is not supported (then the caller uses launch_step).
constexpr int kMaxFuse = 8;

// Synchronisation words of the persistent exp kernel: [0] arrival count,
// [1] generation, [2] error flag, [3] spare, then one epoch word per tile, each
// in its own 32-byte sector (tiles poll their neighbours' words concurrently).
constexpr int kPersistMaxTiles = 4096;
constexpr int kPersistFlagStride = 8;
constexpr size_t kPersistBarWords = 4 + (size_t)kPersistMaxTiles * kPersistFlagStride;
struct FusedStep {
    double tau, gamma_re, gamma_im, rho_re, rho_im;
    int rho_on;
};
// Scalars of one fused pass as the kernels read them.
struct FusedScalars {
    float2 zfac;      // 1 + i s
    float mu;
    float ih2;        // 1 / h^2 (interior coefficient)
    float tau[kMaxFuse];
    float2 gamma[kMaxFuse];
    float2 rho;       // applied after the last step when rho_on
    int rho_on;
};
void fused2d_scalars(int cfg, const FusedStep *steps, float2 zfac, float mu, float ih2, FusedScalars *out);
// Tile plan of configuration cfg on an n0 x n1 grid (tyo <= 0: the largest height).
bool fused2d_tiles(int cfg, int n0, int n1, int tyo, int *txo, int *tyo_out, int *ntx, int *nty);
// One problem of a grouped pass (fused2d.cu): its grid, coefficient table,
// kappa, tile plan, the four batch slots (its sources' vectors n0 * n1 apart)
// and the global index of its first source in the group's active mask.
struct GroupProblem {
    int n0, n1, npml, nmax, txo, tyo;
    const float2 *coef;
    const float *kappa;
    void *slot[4];
    int src0;
};
// One launch of a fused pass over every (problem, source, tile) item of a group:
// bmap[b] = (problem, source of the problem, tile x, tile y); sc_tab[p] = the
// pass scalars of problem p; active[src0 + source] == 0 skips the item.  iv < 0:
// no psi source term.
template <typename S>
bool launch_fused2d_group(int cfg, const GroupProblem *gp, const int4 *bmap, int nblocks,
                          const FusedScalars *sc_tab, const int *active, int iin, int iy, int iv, int iout,
                          cudaStream_t st);
int fused2d_num_cfgs();
int fused2d_cfg_k(int cfg);
int fused2d_cfg_max_tyo(int cfg);
int fused2d_cfg_rx(int cfg);   // largest output-tile height of the configuration
// tyo: output-tile height (<= fused2d_cfg_max_tyo; <= 0 selects the largest)
// nb: batch of vectors of this grid stored n apart (blockIdx.z selects one)
template <typename S>
bool launch_fused2d(int cfg, int tyo, const Geom &g, int npml, const float2 *coef, const float *kappa,
                    const FusedStep *steps, const float2 zfac, float mu, float ih2,
                    const S *pin, const S *y, const S *v, S *pout, cudaStream_t st, int nb = 1);

// Fused 3D sweeps (z-marching temporal blocking, exp actions): see fused3d.cu.
int fused3d_num_cfgs();
int fused3d_cfg_k(int cfg);
template <typename S>
bool launch_fused3d(int cfg, int lz, const Geom &g, const float2 *coef, const float *kappa,
                    const FusedStep *steps, float2 zfac, const S *pin, const S *y, S *pout, cudaStream_t st);

// Persistent exp action (2D, float storage types): see persist2d.cu.
int persist2d_num_cfgs();
int persist2d_cfg_k(int cfg);
// whether configuration cfg adds ghost-point face terms
bool persist2d_cfg_faces(int cfg);
template <typename S>
bool persist2d_plan(int cfg, int n0, int n1, int device, int *txo, int *tyo, int *ntx, int *nty);
template <typename S>
cudaError_t launch_persist2d(int cfg, const Geom &g, int npml, const float2 *coef, const float *kappa,
                             float2 zfac, float h2, const float *tau_dev, int npass,
                             int pass_per_sub, float2 rho, unsigned *bar, int txo, int tyo,
                             int ntx, int nty, const S *x, S *ex0, S *ex1, S *out, cudaStream_t st,
                             const S *w = nullptr, const float2 *wcoef = nullptr,
                             const float2 *const *faces = nullptr);

// Runs the bounded grid barrier with an arrival count that is never reached.
cudaError_t barrier_selftest(unsigned *bar, cudaStream_t st);

template <typename S>
void launch_convert_in(const double2 *x, S *out, int64_t n, cudaStream_t st);
// out = x (mode 0) or out = base - x (mode 1), both complex128
template <typename S>
void launch_convert_out(const S *x, double2 *out, const double2 *base, int mode, int64_t n,
                        cudaStream_t st);

// Krylov kernels (complex128, FP64)
struct KrylovScratch {
    double2 *partials = nullptr;   // [kGridRed][kChunk] block partial sums
    int grid = 0;
};
constexpr int kChunk = 8;
// out[i] (+)= sum_p conj(V_i[p]) w[p] for i < nvec; V_i = V + i * ld.
// gate (nullable, device): when *gate == 0 the launches do nothing.
void krylov_mdot(const double2 *V, int64_t ld, int nvec, const double2 *w, int64_t n,
                 double2 *out, int accumulate, const KrylovScratch &ks, cudaStream_t st,
                 const double *gate = nullptr);
// w += sign * sum_i coef[i] V_i  (coef on the device)
void krylov_maxpy(double2 *w, const double2 *V, int64_t ld, int nvec, const double2 *coef,
                  double sign, int64_t n, cudaStream_t st, const double *gate = nullptr);
// *gate = 1 if the first Gram-Schmidt pass left less than eta of ||w||
// (col[0..j] = projections, col[j+1].x = ||w||^2 before them), else 0.
void krylov_reorth_gate(const double2 *col, int j, double *gate, cudaStream_t st);
// ||w||^2 into *out_dev (device double), deterministic
void krylov_nrm2sq(const double2 *w, int64_t n, double *out_dev, const KrylovScratch &ks,
                   cudaStream_t st);
// w = x * (1 / sqrt(*nrm2sq_dev)) if that is > 0
void krylov_scale_invnorm(double2 *w, const double2 *x, const double *nrm2sq_dev, int64_t n,
                          cudaStream_t st);
// y = x - A-ish helpers
void krylov_sub(double2 *out, const double2 *a, const double2 *b, int64_t n, cudaStream_t st);
void krylov_copy(double2 *out, const double2 *a, int64_t n, cudaStream_t st);
void krylov_add(double2 *out, const double2 *a, int64_t n, cudaStream_t st);   // out += a
void krylov_scale(double2 *w, double2 a, int64_t n, cudaStream_t st);     // w *= a
void krylov_addvec(double2 *a, const double2 *b, int n, cudaStream_t st, const double *gate = nullptr);
// kappa = omega^2 / c^2 in double and float
void compute_kappa(const double *c, double omega, double *k64, float *k32, int64_t n,
                   cudaStream_t st);

// Hessenberg / Givens state on the device for one Arnoldi process.
struct HessState {
    double2 *H;      // (R+1) x R, column-major: H[j*(R+1)+i]
    double *cs;      // R
    double2 *sn;     // R
    double2 *g;      // R+1
    double2 *y;      // R
    double *scal;    // [0] = ||w||^2 of the new vector, [1] = residual estimate |g_{j+1}|,
                     // [2] = breakdown flag, [3] = beta (initial residual norm)
    int R;
};
// After CGS: H[0..j, j] holds the projections; scal[0] holds ||w||^2.
// Sets H[j+1,j], applies/creates rotations, updates g, writes scal[1].
void hess_update(const HessState &hs, int j, cudaStream_t st);
// g = (beta, 0, ...), beta = sqrt(scal[0]); scal[3] = beta.
void hess_start(const HessState &hs, cudaStream_t st);
// Solve the j x j upper-triangular system H y = g into hs.y.
void hess_backsolve(const HessState &hs, int j, cudaStream_t st);

// Tensor-core (tcgen05) forward 3x3 convolution of the learned stage (conv_tc.cu):
// stride S (1 or 2), input nearest-upsampled by 2 when UPS, Cout <= 64;
// *err receives 1 when a bounded wait gives up.  Returns false for an
// unsupported shape.
bool conv_fwd_tc(int S, int UPS, const float *in, int N, int Cin, int Hs, int Ws, const __nv_bfloat16 *w,
                 const float *bias, int Cout, int Ho, int Wo, int relu, const float *skip, float *out,
                 float *out_skip, unsigned *err, cudaStream_t st);

// Tensor-core input gradient of a 3x3 convolution of stride S (conv_tc.cu):
// gin [N][Cin][Hl][Wl] from gout [N][Cout][Ho][Wo] and the layer's weights
// W [Cout][Cin][3][3]; Cin <= 64.
bool conv_bwd_data_tc(int S, const float *gout, int N, int Cout, int Ho, int Wo, const __nv_bfloat16 *w, int Cin,
                      int Hl, int Wl, float *gin, unsigned *err, cudaStream_t st);

// Tensor-core weight gradient of a 3x3 convolution (conv_tc.cu): gw [Cout][Cin * 9]
// = sum over pixels of im2col(x) x g (x the layer input [N][Cin][Hs][Ws], upsampled
// when UPS; g the output gradient [N][Cout][Ho][Wo]); Cout <= 64.  Overwrites gw.
bool conv_wgrad_tc(int S, int UPS, const float *x, int N, int Cin, int Hs, int Ws, const float *g, int Cout, int Ho,
                   int Wo, float *gw, unsigned *err, cudaStream_t st);

// Learned stage: z = network(v) on a 2D grid (n0 x n1), see cnn.cu.
mxp_status cnn_apply_vector(mxp_cnn *net, int n0, int n1, const double2 *v, double vnorm,
                            const double *c, double cmax, double2 *z);

}  // namespace mxp
