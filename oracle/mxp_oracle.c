/*
 * MatExPre CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision restatement of what the MatExPre method
 * computes (arXiv 2506.03617), written from the paper's definitions.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library; the product path never does.  It shares no code, header, table or
 * helper with the CUDA implementation.
 *
 * Contents, each with the passage it follows:
 *   orc_apply     finite-difference Helmholtz operator with PML and complex
 *                 shift (Eq. helmholtz; Eq. pml-1d-s, extended to 2D/3D by
 *                 stretching each axis; shifted operator A_s = A + i w^2 s D of
 *                 Sec. 3.4 "Numerical strategies"); faces zero Dirichlet by
 *                 default, or sound-hard / first-order absorbing through ghost
 *                 points (the mixed boundary conditions of Sec. 4, Marmousi-II).
 *   orc_phi       exp(M)v, psi_1(M)v and psi_2(M)v for M = i t A_s (Def. psi):
 *                 truncated Taylor series over sub-steps.
 *   orc_matexpre  Algorithm 1: r <- psi_1(i t A_s) r, then GMRES on
 *                 (I - exp(i t A_s)) w = r to relative tolerance fprtol
 *                 (Eq. fixed-point), constant -i t dropped (Sec. 3.4).
 *   orc_fgmres    outer flexible GMRES with Algorithm 1 as right preconditioner
 *                 (Sec. 3.4; restart 30 as in Sec. 4).
 *   orc_neumann   truncated Neumann preconditioner P_N of Sec. 3.2 (Thm. 3.1),
 *                 without its constant -i t.
 *   orc_matexpre_v  Algorithm 1 (variant 0) or the same steps on the second
 *                 inverse formula of Sec. 3.1 (variant 1): r <- psi_2(i t A_s) r,
 *                 GMRES on (I - psi_1(i t A_s)) w = r.
 *
 * Grid reading (the paper gives only the 1D operator): unknown j of axis d
 * sits at x_j = (j - npml + 1/2) h, j = 0 .. n_d - 1, n_d = N_d + 2 npml;
 * zero Dirichlet values at j = -1 and j = n_d.  The PML distance is
 * dist = max(0, -x, x - N_d h), delta = npml h, and
 * s(x) = 1 + i Cpml/(delta omega) (dist/delta)^2 (Eq. pml-1d-s).
 * The 2D/3D operator is sum_d (1/s_d) d/dx_d ((1/s_d) d/dx_d u) + omega^2/c^2 u,
 * discretised in flux form with 1/s_d sampled at nodes (outer factor) and at
 * half nodes (inner factor).
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

typedef struct {
    int dim;          /* 2 or 3 */
    int ni[3];        /* interior cells per axis (1 for unused axes) */
    int npml;         /* PML cells on each side */
    double h;         /* mesh size */
    double omega;     /* angular frequency */
    double cpml;      /* PML strength C_pml */
    double shift;     /* complex shift s of A_s */
    double t;         /* time length t */
    const double *c;  /* wave speed at every unknown, x fastest */
    int bc[6];        /* boundary condition of faces x-, x+, y-, y+, z-, z+:
                         0 zero Dirichlet, 1 sound-hard, 2 first-order absorbing */
} orc_problem;

typedef struct {
    int iters;            /* iterations performed */
    int converged;        /* 1 if the tolerance test passed */
    double res_est;       /* last residual estimate (absolute) */
    double res0;          /* initial residual norm */
    int64_t spmv;         /* operator applications spent */
} orc_krylov_stats;

/* ---------- grid helpers ---------- */

static int axis_len(const orc_problem *P, int d)
{
    if (d >= P->dim) return 1;
    return P->ni[d] + 2 * P->npml;
}

static int64_t n_total(const orc_problem *P)
{
    return (int64_t)axis_len(P, 0) * axis_len(P, 1) * axis_len(P, 2);
}

/* 1/s_d at coordinate x (Eq. pml-1d-s). */
static cplx inv_stretch(const orc_problem *P, int d, double x)
{
    if (P->npml == 0) return 1.0;
    double L = P->ni[d] * P->h;
    double delta = P->npml * P->h;
    double dist = 0.0;
    if (x < 0.0) dist = -x;
    if (x > L) dist = x - L;
    double r = dist / delta;
    cplx s = 1.0 + I * (P->cpml / (delta * P->omega)) * r * r;
    return 1.0 / s;
}

static double node_x(const orc_problem *P, int j)
{
    return ((double)j - P->npml + 0.5) * P->h;
}

int64_t orc_n_total(const orc_problem *P) { return n_total(P); }

/* ---------- operator ---------- */

/* 1/s_d at the nodes (a), and at the half nodes x_j + h/2 (bp) and x_j - h/2 (bm). */
static void stretch_arrays(const orc_problem *P, int d, cplx *a, cplx *bp, cplx *bm)
{
    int n = axis_len(P, d);
    for (int j = 0; j < n; ++j) {
        double xq = node_x(P, j);
        a[j] = inv_stretch(P, d, xq);
        bp[j] = inv_stretch(P, d, xq + 0.5 * P->h);
        bm[j] = inv_stretch(P, d, xq - 0.5 * P->h);
    }
}

/*
 * Ghost value at a face (Sec. 4, Marmousi-II: a sound-hard surface and
 * first-order absorbing boundaries [Engquist-Majda], discretised with ghost
 * points).  The boundary lies midway between the last unknown u_0 and its ghost
 * u_g; the face condition, written with the centred difference and the mean
 * there, gives u_g = f u_0 with
 *   zero Dirichlet           u = 0 beyond the grid      f = 0
 *   sound-hard               du/dn = 0                   f = 1
 *   first-order absorbing    du/dn = i k u, k = omega/c_p (outgoing waves for
 *                            the e^{-i omega t} convention)
 *                            (u_g - u_0)/h = i k (u_g + u_0)/2
 *                                            f = (1 + i k h/2) / (1 - i k h/2)
 */
static cplx ghost_factor(const orc_problem *P, int face, double cp)
{
    switch (P->bc[face]) {
    case 1: return 1.0;
    case 2: {
        double kh2 = 0.5 * P->omega / cp * P->h;
        return (1.0 + I * kh2) / (1.0 - I * kh2);
    }
    default: return 0.0;
    }
}

/*
 * y = A x (shifted = 0) or y = A_s x (shifted = 1).
 * (A x)_p = sum_d a_d(x_p) [ b_d(x_p + h/2)(x_{p+e_d} - x_p)
 *                           - b_d(x_p - h/2)(x_p - x_{p-e_d}) ] / h^2
 *           + omega^2 (1 + i s [shifted]) / c_p^2 x_p,
 * with a_d, b_d = 1/s_d; a neighbour beyond the grid is the face's ghost value
 * (zero for the default Dirichlet faces).
 */
void orc_apply(const orc_problem *P, int shifted, const cplx *x, cplx *y)
{
    int n0 = axis_len(P, 0), n1 = axis_len(P, 1), n2 = axis_len(P, 2);
    int64_t stride[3] = {1, n0, (int64_t)n0 * n1};
    int nn[3] = {n0, n1, n2};
    double ih2 = 1.0 / (P->h * P->h);
    double w2 = P->omega * P->omega;
    cplx zfac = shifted ? (1.0 + I * P->shift) : 1.0;
    cplx *a[3], *bp[3], *bm[3];
    for (int d = 0; d < P->dim; ++d) {
        a[d] = malloc(nn[d] * sizeof(cplx));
        bp[d] = malloc(nn[d] * sizeof(cplx));
        bm[d] = malloc(nn[d] * sizeof(cplx));
        stretch_arrays(P, d, a[d], bp[d], bm[d]);
    }

    #pragma omp parallel for schedule(static)
    for (int k = 0; k < n2; ++k) {
        for (int j = 0; j < n1; ++j) {
            for (int i = 0; i < n0; ++i) {
                int idx[3] = {i, j, k};
                int64_t p = i + stride[1] * j + stride[2] * k;
                cplx acc = 0.0;
                double cp = P->c[p];
                for (int d = 0; d < P->dim; ++d) {
                    int q = idx[d];
                    cplx xp = (q + 1 < nn[d]) ? x[p + stride[d]] : ghost_factor(P, 2 * d + 1, cp) * x[p];
                    cplx xm = (q - 1 >= 0) ? x[p - stride[d]] : ghost_factor(P, 2 * d, cp) * x[p];
                    acc += a[d][q] * (bp[d][q] * (xp - x[p]) - bm[d][q] * (x[p] - xm)) * ih2;
                }
                acc += w2 * zfac / (cp * cp) * x[p];
                y[p] = acc;
            }
        }
    }
    for (int d = 0; d < P->dim; ++d) { free(a[d]); free(bp[d]); free(bm[d]); }
}

/* ---------- vector helpers ---------- */

static cplx vdot(int64_t n, const cplx *u, const cplx *v) /* sum conj(u) v */
{
    double re = 0.0, im = 0.0;
    #pragma omp parallel for reduction(+:re,im) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        cplx z = conj(u[i]) * v[i];
        re += creal(z);
        im += cimag(z);
    }
    return re + I * im;
}

static double vnorm(int64_t n, const cplx *u)
{
    double s = 0.0;
    #pragma omp parallel for reduction(+:s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += creal(u[i]) * creal(u[i]) + cimag(u[i]) * cimag(u[i]);
    return sqrt(s);
}

double orc_norm2(int64_t n, const cplx *u) { return vnorm(n, u); }

/* Row-sum (infinity) norm of the matrix t*A_s: max_p sum_q |t A_s(p,q)|. */
double orc_norm_inf_tA(const orc_problem *P, int shifted)
{
    int n0 = axis_len(P, 0), n1 = axis_len(P, 1), n2 = axis_len(P, 2);
    int nn[3] = {n0, n1, n2};
    double ih2 = 1.0 / (P->h * P->h);
    double w2 = P->omega * P->omega;
    cplx zfac = shifted ? (1.0 + I * P->shift) : 1.0;
    double best = 0.0;
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i) {
                int idx[3] = {i, j, k};
                int64_t p = i + (int64_t)n0 * j + (int64_t)n0 * n1 * k;
                cplx diag = w2 * zfac / (P->c[p] * P->c[p]);
                double off = 0.0;
                for (int d = 0; d < P->dim; ++d) {
                    double xq = node_x(P, idx[d]);
                    cplx a = inv_stretch(P, d, xq);
                    cplx bp = inv_stretch(P, d, xq + 0.5 * P->h);
                    cplx bm = inv_stretch(P, d, xq - 0.5 * P->h);
                    diag -= a * (bp + bm) * ih2;
                    if (idx[d] + 1 < nn[d]) off += cabs(a * bp) * ih2;
                    else diag += a * bp * ghost_factor(P, 2 * d + 1, P->c[p]) * ih2;
                    if (idx[d] - 1 >= 0) off += cabs(a * bm) * ih2;
                    else diag += a * bm * ghost_factor(P, 2 * d, P->c[p]) * ih2;
                }
                double row = P->t * (off + cabs(diag));
                if (row > best) best = row;
            }
    return best;
}

/* ---------- matrix functions (Def. psi) ---------- */

/*
 * which = 0: y = exp(M) x;  which = 1: y = psi_1(M) x;  which = 2: y = psi_2(M) x;
 * M = i t A_s (or i t A).
 *
 * The psi functions are solutions of linear ODEs on [0, 1] (Def. psi, through
 * psi_l(z) = int_0^1 exp((1 - s) z) s^(l-1) / (l-1)! ds):
 *   exp(M)x   = u(1) for u' = M u,          u(0) = x;
 *   psi_1(M)x = u(1) for u' = M u + x,      u(0) = 0;
 *   psi_2(M)x = u(1) for u' = M u + tau x,  u(0) = 0.
 * Sub-stepping with step length hs = 1/m_sub and X = hs M: by variation of
 * constants, over the sub-step starting at tau_j = j hs
 *   u <- exp(X) u + hs psi_1(X) g_j + hs^2 psi_2(X) g',
 * where g_j is the forcing at tau_j (x for psi_1, tau_j x for psi_2) and g' its
 * slope (0 for psi_1, x for psi_2).  Each function is its Taylor series:
 * exp(X) z = sum_k X^k z / k!, psi_1(X) z = sum_k X^k z / (k+1)!,
 * psi_2(X) z = sum_k X^k z / (k+2)!.
 * m_sub = ceil(||M||_inf / 2), so ||X|| <= 2 and the Taylor terms shrink at
 * least geometrically once k >= 2; summation stops when the newest terms fall
 * below 1e-17 of the partial sum.
 */
int64_t orc_phi(const orc_problem *P, int which, int shifted, const cplx *x, cplx *y)
{
    int64_t n = n_total(P);
    double nrm = orc_norm_inf_tA(P, shifted);
    int m_sub = (int)ceil(nrm / 2.0);
    if (m_sub < 1) m_sub = 1;
    double inv_m = 1.0 / m_sub;
    cplx xfac = I * P->t * inv_m;       /* X = xfac * A_s */
    int64_t spmv = 0;

    cplx *u = calloc(n, sizeof(cplx));
    cplx *ta = malloc(n * sizeof(cplx));   /* X^k u / k!                   */
    cplx *tb = malloc(n * sizeof(cplx));   /* hs X^k g_j / (k+1)!          */
    cplx *tc = malloc(n * sizeof(cplx));   /* hs^2 X^k g' / (k+2)!         */
    cplx *tmp = malloc(n * sizeof(cplx));
    cplx *next = malloc(n * sizeof(cplx));
    const int has_b = (which >= 1), has_c = (which == 2);
    if (which == 0) memcpy(u, x, n * sizeof(cplx));

    for (int step = 0; step < m_sub; ++step) {
        /* forcing at the sub-step start: x (psi_1) or tau_j x (psi_2) */
        double gj = (which == 1) ? 1.0 : (double)step * inv_m;
        /* k = 0 terms */
        memcpy(ta, u, n * sizeof(cplx));
        for (int64_t i = 0; i < n; ++i) {
            tb[i] = has_b ? x[i] * (gj * inv_m) : 0.0;
            tc[i] = has_c ? x[i] * (inv_m * inv_m / 2.0) : 0.0;
        }
        cplx *acc = tmp;
        for (int64_t i = 0; i < n; ++i) acc[i] = ta[i] + tb[i] + tc[i];
        for (int k = 1; k < 400; ++k) {
            /* ta <- X ta / k */
            orc_apply(P, shifted, ta, next); ++spmv;
            for (int64_t i = 0; i < n; ++i) ta[i] = xfac * next[i] / (double)k;
            double na = vnorm(n, ta), nb = 0.0, nc = 0.0;
            if (has_b) {
                /* tb <- X tb / (k+1) */
                orc_apply(P, shifted, tb, next); ++spmv;
                for (int64_t i = 0; i < n; ++i) tb[i] = xfac * next[i] / (double)(k + 1);
                nb = vnorm(n, tb);
            }
            if (has_c) {
                /* tc <- X tc / (k+2) */
                orc_apply(P, shifted, tc, next); ++spmv;
                for (int64_t i = 0; i < n; ++i) tc[i] = xfac * next[i] / (double)(k + 2);
                nc = vnorm(n, tc);
            }
            for (int64_t i = 0; i < n; ++i) acc[i] += ta[i] + tb[i] + tc[i];
            double ns = vnorm(n, acc);
            if (k >= 3 && na + nb + nc <= 1e-17 * ns) break;
            if (ns == 0.0 && na + nb + nc == 0.0) break;
        }
        memcpy(u, acc, n * sizeof(cplx));
    }
    memcpy(y, u, n * sizeof(cplx));
    free(u); free(ta); free(tb); free(tc); free(tmp); free(next);
    return spmv;
}

/* ---------- flexible GMRES with modified Gram-Schmidt and Givens ---------- */

typedef void (*matvec_fn)(void *ctx, const cplx *in, cplx *out);

/* Complex Givens rotation that zeroes b in (a, b): [c s; -conj(s) c]. */
static void givens(cplx a, cplx b, double *c, cplx *s)
{
    double na = cabs(a), nb = cabs(b);
    if (nb == 0.0) { *c = 1.0; *s = 0.0; return; }
    if (na == 0.0) { *c = 0.0; *s = conj(b) / nb; return; }
    double r = hypot(na, nb);
    *c = na / r;
    *s = (a / na) * conj(b) / r;
}

/*
 * Solve A x = b by restarted flexible GMRES (right preconditioning z = M^-1 v;
 * precond == NULL means z = v, i.e. plain GMRES).  x holds the initial guess on
 * entry.  Stops when the least-squares residual estimate is <= tol_abs; if
 * fixed > 0 the tolerance is ignored and exactly `fixed` iterations are taken.
 * On a restart (and at the end when check_true is set) the true residual
 * b - A x is recomputed; with check_true the solve only counts as converged
 * once that true residual is <= tol_abs.
 */
static void fgmres_core(int64_t n, matvec_fn A, void *actx, matvec_fn Minv, void *mctx,
                        const cplx *b, cplx *x, double tol_abs, int restart, int maxit,
                        int fixed, int check_true, orc_krylov_stats *st,
                        double *res_log)
{
    cplx *V = malloc((size_t)(restart + 1) * n * sizeof(cplx));
    cplx *Z = Minv ? malloc((size_t)restart * n * sizeof(cplx)) : NULL;
    cplx *Hm = calloc((size_t)(restart + 1) * restart, sizeof(cplx)); /* H[i][j] at i*restart+j */
    double *cs = malloc(restart * sizeof(double));
    cplx *sn = malloc(restart * sizeof(cplx));
    cplx *g = malloc((restart + 1) * sizeof(cplx));
    cplx *yv = malloc(restart * sizeof(cplx));
    cplx *w = malloc(n * sizeof(cplx));
    int total = 0;
    int target = fixed > 0 ? fixed : maxit;
    st->converged = 0;
    st->spmv = 0;

    /* r0 = b - A x */
    A(actx, x, w); st->spmv++;
    for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
    double beta = vnorm(n, w);
    st->res0 = beta;
    st->res_est = beta;
    if (fixed <= 0 && beta <= tol_abs) { st->converged = 1; goto done; }

    while (total < target) {
        if (beta == 0.0) { st->converged = 1; break; }
        for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(g, 0, (restart + 1) * sizeof(cplx));
        memset(Hm, 0, (size_t)(restart + 1) * restart * sizeof(cplx));
        g[0] = beta;
        int j = 0, stop = 0;
        for (; j < restart && total < target; ++j) {
            cplx *vj = V + (size_t)j * n;
            const cplx *zj = vj;
            if (Minv) { Minv(mctx, vj, Z + (size_t)j * n); zj = Z + (size_t)j * n; }
            cplx *vn = V + (size_t)(j + 1) * n;
            A(actx, zj, vn); st->spmv++;
            for (int i = 0; i <= j; ++i) {   /* modified Gram-Schmidt */
                cplx *vi = V + (size_t)i * n;
                cplx hij = vdot(n, vi, vn);
                Hm[i * restart + j] = hij;
                for (int64_t q = 0; q < n; ++q) vn[q] -= hij * vi[q];
            }
            double hn = vnorm(n, vn);
            Hm[(j + 1) * restart + j] = hn;
            if (hn > 0.0) for (int64_t q = 0; q < n; ++q) vn[q] /= hn;
            for (int i = 0; i < j; ++i) {    /* previous rotations */
                cplx a = Hm[i * restart + j], bb = Hm[(i + 1) * restart + j];
                Hm[i * restart + j] = cs[i] * a + sn[i] * bb;
                Hm[(i + 1) * restart + j] = -conj(sn[i]) * a + cs[i] * bb;
            }
            givens(Hm[j * restart + j], Hm[(j + 1) * restart + j], &cs[j], &sn[j]);
            cplx a = Hm[j * restart + j], bb = Hm[(j + 1) * restart + j];
            Hm[j * restart + j] = cs[j] * a + sn[j] * bb;
            Hm[(j + 1) * restart + j] = 0.0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            st->res_est = cabs(g[j + 1]);
            if (res_log) res_log[total - 1] = st->res_est;
            if (hn == 0.0) { stop = 1; ++j; break; }           /* happy breakdown */
            if (fixed <= 0 && st->res_est <= tol_abs) { stop = 1; ++j; break; }
        }
        /* back-substitution H y = g, then x += Z y (or V y) */
        for (int i = j - 1; i >= 0; --i) {
            cplx s = g[i];
            for (int k = i + 1; k < j; ++k) s -= Hm[i * restart + k] * yv[k];
            yv[i] = s / Hm[i * restart + i];
        }
        for (int i = 0; i < j; ++i) {
            const cplx *zi = Minv ? Z + (size_t)i * n : V + (size_t)i * n;
            for (int64_t q = 0; q < n; ++q) x[q] += yv[i] * zi[q];
        }
        int need_true = (!stop && total < target) || check_true;
        if (need_true) {
            A(actx, x, w); st->spmv++;
            for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
            beta = vnorm(n, w);
            st->res_est = beta;
            if (fixed <= 0 && beta <= tol_abs) { st->converged = 1; break; }
            if (stop && beta == 0.0) { st->converged = 1; break; }
        } else if (stop) {
            st->converged = 1;
            break;
        }
        if (stop && !check_true) break;
    }
done:
    st->iters = total;
    free(V); free(Z); free(Hm); free(cs); free(sn); free(g); free(yv); free(w);
}

/* ---------- Algorithm 1 ---------- */

typedef struct {
    const orc_problem *P;
    int which;          /* 0: exp (Algorithm 1), 1: psi_1 (second inverse formula) */
    int64_t spmv;
} fp_ctx;

/* out = (I - phi(i t A_s)) in, phi = exp (Eq. fixed-point) or psi_1 */
static void fixed_point_op(void *vctx, const cplx *in, cplx *out)
{
    fp_ctx *c = vctx;
    int64_t n = n_total(c->P);
    c->spmv += orc_phi(c->P, c->which, 1, in, out);
    for (int64_t i = 0; i < n; ++i) out[i] = in[i] - out[i];
}

/*
 * variant 0, Algorithm 1: r <- psi_1(i t A_s) r; zeta = ||r||; GMRES(restart),
 * x0 = 0, on (I - exp(i t A_s)) w = r until the residual estimate is
 * <= fprtol * zeta (or exactly `fixed` iterations when fixed > 0, or maxit).
 * variant 1, the same steps on the second inverse formula of Sec. 3.1,
 * A^{-1} = -i t (I - psi_1(i t A))^{-1} psi_2(i t A): r <- psi_2(i t A_s) r and
 * GMRES on (I - psi_1(i t A_s)) w = r.  Both give w ~ (i/t) A_s^{-1} r.
 * Returns the number of inner iterations; *spmv_out gets the operator count.
 */
int orc_matexpre_v(const orc_problem *P, int variant, const cplx *r, cplx *w, double fprtol,
                   int restart, int maxit, int fixed, int64_t *spmv_out)
{
    int64_t n = n_total(P);
    cplx *rt = malloc(n * sizeof(cplx));
    fp_ctx ctx = {P, variant == 1 ? 1 : 0, 0};
    ctx.spmv += orc_phi(P, variant == 1 ? 2 : 1, 1, r, rt);
    double zeta = vnorm(n, rt);
    memset(w, 0, n * sizeof(cplx));
    orc_krylov_stats st;
    fgmres_core(n, fixed_point_op, &ctx, NULL, NULL, rt, w, fprtol * zeta, restart,
                maxit, fixed, 0, &st, NULL);
    free(rt);
    if (spmv_out) *spmv_out = ctx.spmv;
    return st.iters;
}

int orc_matexpre(const orc_problem *P, const cplx *r, cplx *w, double fprtol,
                 int restart, int maxit, int fixed, int64_t *spmv_out)
{
    return orc_matexpre_v(P, 0, r, w, fprtol, restart, maxit, fixed, spmv_out);
}

/*
 * Truncated Neumann preconditioner of Sec. 3.2 without its constant -i t:
 * w = (sum_{n=0}^{N} exp(i t A_s)^n) psi_1(i t A_s) r.
 */
int64_t orc_neumann(const orc_problem *P, int shifted, int nterms, const cplx *r, cplx *w)
{
    int64_t n = n_total(P);
    cplx *z = malloc(n * sizeof(cplx));
    cplx *tmp = malloc(n * sizeof(cplx));
    int64_t spmv = orc_phi(P, 1, shifted, r, z);
    memcpy(w, z, n * sizeof(cplx));
    for (int k = 1; k <= nterms; ++k) {
        spmv += orc_phi(P, 0, shifted, z, tmp);
        memcpy(z, tmp, n * sizeof(cplx));
        for (int64_t i = 0; i < n; ++i) w[i] += z[i];
    }
    free(z);
    free(tmp);
    return spmv;
}

/* ---------- outer FGMRES ---------- */

typedef struct {
    const orc_problem *P;
    double fprtol;
    int inner_restart, inner_maxit, inner_fixed;
    int64_t spmv;
    int calls;
    int *inner_log;
    int log_cap;
    int variant;        /* preconditioner variant of orc_matexpre_v */
} outer_ctx;

static void helmholtz_op(void *vctx, const cplx *in, cplx *out)
{
    outer_ctx *c = vctx;
    orc_apply(c->P, 0, in, out);
    c->spmv++;
}

static void matexpre_op(void *vctx, const cplx *in, cplx *out)
{
    outer_ctx *c = vctx;
    int64_t sp = 0;
    int it = orc_matexpre_v(c->P, c->variant, in, out, c->fprtol, c->inner_restart,
                            c->inner_maxit, c->inner_fixed, &sp);
    c->spmv += sp;
    if (c->inner_log && c->calls < c->log_cap) c->inner_log[c->calls] = it;
    c->calls++;
}

typedef struct {
    int outer_iters;
    int converged;
    double true_relres;
    double est_relres;
    int64_t spmv;
} orc_solve_stats;

/*
 * Solve A u = b (unshifted A) by FGMRES(restart) with Algorithm 1 as the right
 * preconditioner.  u holds the initial guess on entry (zero for the paper's
 * runs).  Stops when the estimate is <= rtol ||b|| and the recomputed true
 * residual confirms it; restarts otherwise, up to maxit outer iterations.
 * inner_log (nullable, capacity log_cap) receives the inner iteration count of
 * every preconditioner application; res_log (nullable, capacity maxit) gets
 * the residual estimate after every outer iteration.
 */
void orc_fgmres_v(const orc_problem *P, int variant, const cplx *b, cplx *u, double rtol,
                  int restart, int maxit, double fprtol, int inner_restart, int inner_maxit,
                  int inner_fixed, int *inner_log, int log_cap, double *res_log,
                  orc_solve_stats *out)
{
    int64_t n = n_total(P);
    outer_ctx ctx = {P, fprtol, inner_restart, inner_maxit, inner_fixed, 0, 0, inner_log, log_cap,
                     variant};
    double bn = vnorm(n, b);
    orc_krylov_stats st;
    fgmres_core(n, helmholtz_op, &ctx, matexpre_op, &ctx, b, u, rtol * bn, restart, maxit,
                0, 1, &st, res_log);
    cplx *r = malloc(n * sizeof(cplx));
    orc_apply(P, 0, u, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    out->true_relres = bn > 0 ? vnorm(n, r) / bn : 0.0;
    out->est_relres = bn > 0 ? st.res_est / bn : 0.0;
    out->outer_iters = st.iters;
    out->converged = st.converged && out->true_relres <= rtol;
    out->spmv = ctx.spmv + st.spmv + 1;
    free(r);
}

void orc_fgmres(const orc_problem *P, const cplx *b, cplx *u, double rtol, int restart,
                int maxit, double fprtol, int inner_restart, int inner_maxit,
                int inner_fixed, int *inner_log, int log_cap, double *res_log,
                orc_solve_stats *out)
{
    orc_fgmres_v(P, 0, b, u, rtol, restart, maxit, fprtol, inner_restart, inner_maxit,
                 inner_fixed, inner_log, log_cap, res_log, out);
}

/* Plain GMRES on A_s or A (no preconditioner), used by tests as a reference
 * Krylov solve on tiny grids. */
static void op_plain(void *vctx, const cplx *in, cplx *out)
{
    const orc_problem *P = ((void **)vctx)[0];
    int shifted = *(int *)((void **)vctx)[1];
    orc_apply(P, shifted, in, out);
}

int orc_gmres_plain(const orc_problem *P, int shifted, const cplx *b, cplx *x, double rtol,
                    int restart, int maxit)
{
    int64_t n = n_total(P);
    void *ctx[2] = {(void *)P, &shifted};
    orc_krylov_stats st;
    fgmres_core(n, op_plain, ctx, NULL, NULL, b, x, rtol * vnorm(n, b), restart, maxit, 0, 1,
                &st, NULL);
    return st.converged ? st.iters : -st.iters;
}

/* Threads of the parallel loops above (timing runs only; results do not
 * depend on it beyond the order of the reductions' partial sums). */
void orc_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
}
