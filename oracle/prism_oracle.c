/*
 * prism_oracle.c -- plain FP64 CPU oracle of the PRISM QP projection.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may call this library.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.  Everything here is dense, unfused and in the order the paper
 * writes it, so it can be checked against the paper by eye; speed is not a goal.
 *
 * What it computes (paper: Sec. III-D "Custom QP Solver"):
 *   the projection of a sampled joint-velocity sequence xi (one joint; the QP is
 *   separable across joints, Sec. III-D "Joint-wise separability") onto
 *     { x :  G x <= h,  x_1 = thetadot_init }                  Eq. (compact_qp)
 *   with G, h the verbatim stacked operator of Eq. (G_h_def) built from
 *   Eqs. (vel_bounds), (pos_stack), (pos_bounds), (acc_stack), (b_acc),
 *   (acc_bounds), (jerk_stack), (D2_def), (b_jerk), (jerk_bounds) and
 *   A = [1 0 ... 0], b = thetadot_init of Eq. (A_b_def).
 *
 * Two iterations are provided:
 *   ORACLE_MODE_PAPER  the printed scheme, Eqs. (admm_zeta), (admm_primal),
 *                      (admm_KKT), (admm_dual), step factor delta/2 included,
 *                      with the full (H+1)x(H+1) KKT matrix M factored by LDL^T.
 *   ORACLE_MODE_ADMM   the same three steps in the same order (slack clip ->
 *                      KKT solve with the cached factor -> multiplier update)
 *                      but with the multiplier u kept in constraint space and
 *                      seen by the slack step (textbook scaled ADMM on the
 *                      two-sided form lo <= F x <= hi, where F are the "+" rows
 *                      of G).  This reading is used because the printed
 *                      iteration does not converge to the projection that
 *                      Sec. III-D says it computes.
 * Row scaling ORACLE_SCALE_ROWNORM divides every constraint row and its bound by
 * the row's Euclidean norm (the paper is silent on scaling; the feasible set
 * and hence the projection are unchanged).  ORACLE_SCALE_NONE uses G as printed.
 *
 * Initial state (the paper does not state it): x^0 = xi with x^0_1 := v0,
 * and a zero multiplier, unless a warm start is passed in.
 *
 * Pinning (tests/test_oracle_pins.py): G and h against the printed matrices at
 * H=3; the feasible set against its derivative definition; the ADMM limit
 * against brute-force active-set enumeration (H<=5), the H=2 closed form, KKT
 * certificates, idempotence, non-expansiveness and row-scaling invariance; the
 * first primal step of both modes against its argmin definition (least
 * squares); every ADMM iteration against the dual feasibility of scaled ADMM
 * (x - xi + rho F'^T u in span(e1)) and its slack against the box projection
 * (normal-cone condition); the residuals against their definitions; the
 * PAPER fixed point against its stationarity relation, and every PAPER
 * iteration against the stationarity of its primal step combined with the
 * multiplier step (x^{l+1} - xi + lambda^l - 2 lambda^{l+1} in span(e1), which
 * fixes the factor delta/2 of Eq. admm_dual).  Planted mistakes in a copy of
 * this file each fail a pin (tests/test_oracle_mutations.py).
 *
 * Residuals reported per column:
 *   primal = max( |x_1 - v0|, max_r max(0, (G x - h)_r) / ||G_r||_2 )
 *            (row-normalised bound violation of the final iterate, unscaled G)
 *   dual   = max_i |x^L_i - x^{L-1}_i|  (size of the last primal step; 0 if L=0)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_MODE_ADMM = 0, ORACLE_MODE_PAPER = 1 };
enum { ORACLE_SCALE_ROWNORM = 0, ORACLE_SCALE_NONE = 1 };

/* bounds vector order: q_min q_max v_min v_max a_min a_max j_min j_max */
#define QMIN 0
#define QMAX 1
#define VMIN 2
#define VMAX 3
#define AMIN 4
#define AMAX 5
#define JMIN 6
#define JMAX 7

/* ---------------------------------------------------------------------------
 * Eq. (G_h_def) for one joint (N_dof = 1).  G is (8H-2) x H row-major, h has
 * 8H-2 entries.  Block order as printed:
 *   [ I; -I; dt L; -dt L; D1/dt; -D1/dt; D2/dt^2; -D2/dt^2 ]
 *   [ v_max; -v_min; q_max-q0; -(q_min-q0); a_max-b_acc; -a_min+b_acc;
 *     j_max-b_jerk; -j_min+b_jerk ]
 * L: inclusive lower-triangular cumulative sum (Eq. pos_stack);
 * D1: 1 on the diagonal, -1 on the sub-diagonal (Eq. acc_stack);
 * D2: (H-1) x H, first row [-2 1 0 ...], then rows [.. 1 -2 1 ..] (Eq. D2_def);
 * b_acc  = (1/dt)   (-v0, 0, ..., 0)  (Eq. b_acc),  H entries;
 * b_jerk = (1/dt^2) ( v0, 0, ..., 0)  (Eq. b_jerk), H-1 entries.
 * ------------------------------------------------------------------------- */
int oracle_build_G_h(int H, double dt, const double *bnd, double q0, double v0,
                     double *G, double *h)
{
    if (H < 2 || !(dt > 0.0)) return -1;
    const int m = 8 * H - 2;
    memset(G, 0, sizeof(double) * (size_t)m * (size_t)H);
    double *D1 = calloc((size_t)H * H, sizeof(double));
    double *D2 = calloc((size_t)(H - 1) * H, sizeof(double));
    double *L = calloc((size_t)H * H, sizeof(double));
    double *bacc = calloc((size_t)H, sizeof(double));
    double *bjerk = calloc((size_t)(H - 1), sizeof(double));
    if (!D1 || !D2 || !L || !bacc || !bjerk) {
        free(D1); free(D2); free(L); free(bacc); free(bjerk);
        return -2;
    }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j <= i; ++j) L[i * H + j] = 1.0;
    for (int i = 0; i < H; ++i) {
        D1[i * H + i] = 1.0;
        if (i > 0) D1[i * H + i - 1] = -1.0;
    }
    for (int i = 0; i < H - 1; ++i) {
        if (i > 0) D2[i * H + i - 1] = 1.0;
        D2[i * H + i] = -2.0;
        D2[i * H + i + 1] = 1.0;
    }
    bacc[0] = -v0 / dt;
    bjerk[0] = v0 / (dt * dt);

    int r = 0;
    for (int i = 0; i < H; ++i, ++r) { G[r * H + i] = 1.0;  h[r] = bnd[VMAX]; }
    for (int i = 0; i < H; ++i, ++r) { G[r * H + i] = -1.0; h[r] = -bnd[VMIN]; }
    for (int i = 0; i < H; ++i, ++r) {
        for (int j = 0; j < H; ++j) G[r * H + j] = dt * L[i * H + j];
        h[r] = bnd[QMAX] - q0;
    }
    for (int i = 0; i < H; ++i, ++r) {
        for (int j = 0; j < H; ++j) G[r * H + j] = -dt * L[i * H + j];
        h[r] = -(bnd[QMIN] - q0);
    }
    for (int i = 0; i < H; ++i, ++r) {
        for (int j = 0; j < H; ++j) G[r * H + j] = D1[i * H + j] / dt;
        h[r] = bnd[AMAX] - bacc[i];
    }
    for (int i = 0; i < H; ++i, ++r) {
        for (int j = 0; j < H; ++j) G[r * H + j] = -D1[i * H + j] / dt;
        h[r] = -bnd[AMIN] + bacc[i];
    }
    for (int i = 0; i < H - 1; ++i, ++r) {
        for (int j = 0; j < H; ++j) G[r * H + j] = D2[i * H + j] / (dt * dt);
        h[r] = bnd[JMAX] - bjerk[i];
    }
    for (int i = 0; i < H - 1; ++i, ++r) {
        for (int j = 0; j < H; ++j) G[r * H + j] = -D2[i * H + j] / (dt * dt);
        h[r] = -bnd[JMIN] + bjerk[i];
    }
    free(D1); free(D2); free(L); free(bacc); free(bjerk);
    return (r == m) ? 0 : -3;
}

/* Index of the k-th "+" row (k = 0..4H-2) of G: blocks 0, 2, 4, 6. */
static int plus_row(int H, int k)
{
    if (k < H) return k;                       /* velocity   */
    if (k < 2 * H) return 2 * H + (k - H);     /* position   */
    if (k < 3 * H) return 4 * H + (k - 2 * H); /* accel      */
    return 6 * H + (k - 3 * H);                /* jerk       */
}
/* Its "-" partner: the next block. */
static int minus_row(int H, int k)
{
    if (k < H) return H + k;
    if (k < 2 * H) return 3 * H + (k - H);
    if (k < 3 * H) return 5 * H + (k - 2 * H);
    return 6 * H + (H - 1) + (k - 3 * H);
}

/* ---------------------------------------------------------------------------
 * Dense LDL^T (unit lower L, diagonal D) of a symmetric n x n matrix, in
 * place: D on the diagonal, L strictly below.  No pivoting: the KKT matrices
 * here are [[B, e1], [e1^T, 0]] with B symmetric positive definite, whose
 * leading pivots are those of B and whose last pivot is -e1^T B^{-1} e1 < 0.
 * ------------------------------------------------------------------------- */
static int ldlt_factor(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k] * A[k * n + k];
        if (d == 0.0 || !isfinite(d)) return -1;
        A[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k] * A[k * n + k];
            A[i * n + j] = s / d;
        }
    }
    /* mirror L into the upper triangle is not needed: solves read below-diagonal */
    return 0;
}

static void ldlt_solve(int n, const double *A, double *b)
{
    for (int i = 0; i < n; ++i) {              /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= A[i * n + k] * b[k];
        b[i] = s;
    }
    for (int i = 0; i < n; ++i) b[i] /= A[i * n + i];   /* D z = y */
    for (int i = n - 1; i >= 0; --i) {        /* L^T x = z */
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= A[k * n + i] * b[k];
        b[i] = s;
    }
}

/* ---------------------------------------------------------------------------
 * Per-shape set-up shared by all columns of one (H, dt, rho, mode, scale):
 * the scaled operator and the LDL^T factor of its KKT matrix
 * (Sec. III-D "Pre-computable factorization").
 * ------------------------------------------------------------------------- */
typedef struct {
    int H, m, p, mode, scale;
    double dt, rho;
    double *G0;    /* m x H unscaled G (for h and residuals)                 */
    double *gn;    /* m: ||G_r||_2                                           */
    double *Gs;    /* PAPER: m x H scaled G'   (rows G_r * s_r)              */
    double *Fs;    /* ADMM:  p x H scaled F'   ("+" rows, times s_r)         */
    double *fs;    /* ADMM:  p row scales s_r                                */
    double *M;     /* (H+1)^2 LDL^T factor of the KKT matrix                 */
} setup_t;

static void setup_free(setup_t *S)
{
    free(S->G0); free(S->gn); free(S->Gs); free(S->Fs); free(S->fs); free(S->M);
    memset(S, 0, sizeof(*S));
}

static int setup_make(setup_t *S, int mode, int scale, int H, double dt, double rho)
{
    memset(S, 0, sizeof(*S));
    S->H = H; S->m = 8 * H - 2; S->p = 4 * H - 1; S->mode = mode; S->scale = scale;
    S->dt = dt; S->rho = rho;
    const int m = S->m, p = S->p, n = H + 1;
    S->G0 = calloc((size_t)m * H, sizeof(double));
    S->gn = calloc((size_t)m, sizeof(double));
    S->Gs = calloc((size_t)m * H, sizeof(double));
    S->Fs = calloc((size_t)p * H, sizeof(double));
    S->fs = calloc((size_t)p, sizeof(double));
    S->M = calloc((size_t)n * n, sizeof(double));
    double *hdummy = calloc((size_t)m, sizeof(double));
    const double zb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (!S->G0 || !S->gn || !S->Gs || !S->Fs || !S->fs || !S->M || !hdummy) {
        free(hdummy); setup_free(S); return -2;
    }
    if (oracle_build_G_h(H, dt, zb, 0.0, 0.0, S->G0, hdummy) != 0) {
        free(hdummy); setup_free(S); return -1;
    }
    free(hdummy);
    for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int j = 0; j < H; ++j) s += S->G0[r * H + j] * S->G0[r * H + j];
        S->gn[r] = sqrt(s);
    }
    for (int r = 0; r < m; ++r) {
        double sr = (scale == ORACLE_SCALE_ROWNORM) ? 1.0 / S->gn[r] : 1.0;
        for (int j = 0; j < H; ++j) S->Gs[r * H + j] = S->G0[r * H + j] * sr;
    }
    for (int k = 0; k < p; ++k) {
        int r = plus_row(H, k);
        double sr = (scale == ORACLE_SCALE_ROWNORM) ? 1.0 / S->gn[r] : 1.0;
        S->fs[k] = sr;
        for (int j = 0; j < H; ++j) S->Fs[k * H + j] = S->G0[r * H + j] * sr;
    }
    /* KKT matrix M = [[I + c, A^T], [A, 0]], A = e1^T (Eq. admm_primal):
     *   PAPER: c = rho * G'^T G'   (all 8H-2 rows)
     *   ADMM:  c = rho * F'^T F'   (the 4H-1 "+" rows)                       */
    double *Mm = S->M;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < H; ++j) {
            double s = 0.0;
            if (mode == ORACLE_MODE_PAPER) {
                for (int r = 0; r < m; ++r) s += S->Gs[r * H + i] * S->Gs[r * H + j];
            } else {
                for (int k = 0; k < p; ++k) s += S->Fs[k * H + i] * S->Fs[k * H + j];
            }
            Mm[i * n + j] = rho * s + (i == j ? 1.0 : 0.0);
        }
    Mm[0 * n + H] = 1.0;
    Mm[H * n + 0] = 1.0;
    Mm[H * n + H] = 0.0;
    if (ldlt_factor(n, Mm) != 0) { setup_free(S); return -4; }
    return 0;
}

/* K = [M^{-1}]_{1:H,1:H}, kb = [M^{-1}]_{1:H,H+1}: the maps with
 * x^{l+1} = K r_{1:H} + kb * b of Eq. (admm_primal). */
int oracle_kkt_inverse(int mode, int scale, int H, double dt, double rho, double *K, double *kb)
{
    setup_t S;
    int rc = setup_make(&S, mode, scale, H, dt, rho);
    if (rc) return rc;
    const int n = H + 1;
    double *e = malloc(sizeof(double) * n);
    if (!e) { setup_free(&S); return -2; }
    for (int c = 0; c < n; ++c) {
        memset(e, 0, sizeof(double) * n);
        e[c] = 1.0;
        ldlt_solve(n, S.M, e);
        for (int i = 0; i < H; ++i) {
            if (c < H) K[i * H + c] = e[i];
            else kb[i] = e[i];
        }
    }
    free(e);
    setup_free(&S);
    return 0;
}

static double clipd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Primal residual of x against unscaled G x <= h and x_1 = v0. */
static double primal_residual(const setup_t *S, const double *h, const double *x, double v0)
{
    const int H = S->H, m = S->m;
    double res = fabs(x[0] - v0);
    for (int r = 0; r < m; ++r) {
        double g = 0.0;
        for (int j = 0; j < H; ++j) g += S->G0[r * H + j] * x[j];
        double v = (g - h[r]) / S->gn[r];
        if (v > res) res = v;
    }
    return res;
}

/* ---------------------------------------------------------------------------
 * One column.  xi, x (in: warm start or NULL; out: x^L), dual state
 * (ADMM: u' in R^{4H-1}, the multiplier of the scaled rows; PAPER: lambda in
 * R^H) in/out.  work must hold 6*(8H) doubles.
 * ------------------------------------------------------------------------- */
static void solve_column(const setup_t *S, const double *bnd, double q0, double v0,
                         const double *xi, int iters, const double *x_init,
                         const double *dual_init, double *x, double *dual,
                         double *primal, double *dualres, double *work)
{
    const int H = S->H, m = S->m, p = S->p, n = H + 1;
    const double rho = S->rho;
    double *h = work;              /* m   unscaled h                       */
    double *hs = h + m;            /* m   scaled h' (PAPER)                */
    double *lo = hs + m;           /* p   scaled lo' (ADMM)                */
    double *hi = lo + p;           /* p   scaled hi' (ADMM)                */
    double *z = hi + p;            /* m   slack / clipped rows             */
    double *rhs = z + m;           /* n   KKT right-hand side              */
    double *xprev = rhs + n;       /* H                                    */
    double *G0 = malloc(sizeof(double) * (size_t)m * H);
    oracle_build_G_h(H, S->dt, bnd, q0, v0, G0, h);
    free(G0);

    /* x_1 is the boundary value (Eq. proj_boundary) in every iterate, the
     * starting one included: a warm start's first step is replaced by v0 */
    for (int i = 0; i < H; ++i) x[i] = x_init ? x_init[i] : xi[i];
    x[0] = v0;
    memcpy(xprev, x, sizeof(double) * H);

    if (S->mode == ORACLE_MODE_PAPER) {
        double *lam = dual;                                   /* lambda in R^H */
        for (int i = 0; i < H; ++i) lam[i] = dual_init ? dual_init[i] : 0.0;
        for (int r = 0; r < m; ++r) {
            double sr = (S->scale == ORACLE_SCALE_ROWNORM) ? 1.0 / S->gn[r] : 1.0;
            hs[r] = h[r] * sr;
        }
        for (int l = 0; l < iters; ++l) {
            memcpy(xprev, x, sizeof(double) * H);
            /* Step 1, Eq. (admm_zeta): zeta = max(0, -G' x^l + h') */
            for (int r = 0; r < m; ++r) {
                double g = 0.0;
                for (int j = 0; j < H; ++j) g += S->Gs[r * H + j] * x[j];
                double v = -g + hs[r];
                z[r] = v > 0.0 ? v : 0.0;
            }
            /* Step 2, Eqs. (admm_primal), (admm_KKT):
             *   r = [rho G'^T (h' - zeta) + lambda^l + xi ; b],  x = [M^{-1} r]_{1:H} */
            for (int i = 0; i < H; ++i) {
                double s = 0.0;
                for (int r = 0; r < m; ++r) s += S->Gs[r * H + i] * (hs[r] - z[r]);
                rhs[i] = rho * s + lam[i] + xi[i];
            }
            rhs[H] = v0;
            ldlt_solve(n, S->M, rhs);
            for (int i = 0; i < H; ++i) x[i] = rhs[i];
            /* Step 3, Eq. (admm_dual):
             *   lambda -= (rho/2) G'^T (G' x^{l+1} - h' + zeta^{l+1})            */
            /* z now becomes the residual G' x^{l+1} - h' + zeta^{l+1} */
            for (int r = 0; r < m; ++r) {
                double g = 0.0;
                for (int j = 0; j < H; ++j) g += S->Gs[r * H + j] * x[j];
                z[r] = g - hs[r] + z[r];
            }
            for (int i = 0; i < H; ++i) {
                double s = 0.0;
                for (int r = 0; r < m; ++r) s += S->Gs[r * H + i] * z[r];
                lam[i] -= 0.5 * rho * s;
            }
        }
    } else {
        double *u = dual;                                     /* u' in R^{4H-1} */
        for (int k = 0; k < p; ++k) u[k] = dual_init ? dual_init[k] : 0.0;
        for (int k = 0; k < p; ++k) {
            hi[k] = h[plus_row(H, k)] * S->fs[k];
            lo[k] = -h[minus_row(H, k)] * S->fs[k];
        }
        for (int l = 0; l < iters; ++l) {
            memcpy(xprev, x, sizeof(double) * H);
            /* Slack step (counterpart of Eq. admm_zeta): z = clip(F' x^l + u^l, lo', hi') */
            for (int k = 0; k < p; ++k) {
                double g = 0.0;
                for (int j = 0; j < H; ++j) g += S->Fs[k * H + j] * x[j];
                z[k] = clipd(g + u[k], lo[k], hi[k]);
            }
            /* Primal step (counterpart of Eqs. admm_primal, admm_KKT):
             *   [[I + rho F'^T F', e1], [e1^T, 0]] [x; nu] = [xi + rho F'^T (z - u^l); v0] */
            for (int i = 0; i < H; ++i) {
                double s = 0.0;
                for (int k = 0; k < p; ++k) s += S->Fs[k * H + i] * (z[k] - u[k]);
                rhs[i] = xi[i] + rho * s;
            }
            rhs[H] = v0;
            ldlt_solve(n, S->M, rhs);
            for (int i = 0; i < H; ++i) x[i] = rhs[i];
            /* Multiplier step (counterpart of Eq. admm_dual): u += F' x^{l+1} - z */
            for (int k = 0; k < p; ++k) {
                double g = 0.0;
                for (int j = 0; j < H; ++j) g += S->Fs[k * H + j] * x[j];
                u[k] += g - z[k];
            }
        }
    }
    double d = 0.0;
    if (iters > 0)
        for (int i = 0; i < H; ++i) {
            double a = fabs(x[i] - xprev[i]);
            if (a > d) d = a;
        }
    *dualres = d;
    *primal = primal_residual(S, h, x, v0);
}

/* ---------------------------------------------------------------------------
 * A batch of N samples x J joints in the paper's stacking [N][H][J]
 * (time-major, joint-minor; Sec. III-D "From Joint-Velocity Sequences ...").
 *   bounds   [8][J]
 *   q0, v0   [J]
 *   xi       [N][H][J]
 *   x_init   [N][H][J] or NULL (its first step is replaced by v0);
 *            dual_init [N][D][J] or NULL,
 *            D = 4H-1 (ADMM, scaled multiplier u') or H (PAPER, lambda)
 *   x_out    [N][H][J];  primal, dual [N][J];  dual_out [N][D][J] or NULL
 *   cols     optional list of flattened columns n*J + j to solve (others are
 *            left untouched); NULL solves all N*J columns.
 * Returns 0 on success.
 * ------------------------------------------------------------------------- */
int oracle_solve_batch(int mode, int scale, int N, int J, int H, double dt,
                       const double *bounds, const double *q0, const double *v0,
                       const double *xi, int iters, double rho,
                       const double *x_init, const double *dual_init,
                       double *x_out, double *primal, double *dual, double *dual_out,
                       const long long *cols, long long ncols, int nthreads)
{
    if (N < 0 || J <= 0 || H < 2 || !(dt > 0.0) || iters < 0 || !(rho > 0.0)) return -1;
    if (mode != ORACLE_MODE_ADMM && mode != ORACLE_MODE_PAPER) return -1;
    if (scale != ORACLE_SCALE_ROWNORM && scale != ORACLE_SCALE_NONE) return -1;
    setup_t S;
    int rc = setup_make(&S, mode, scale, H, dt, rho);
    if (rc) return rc;
    const int D = (mode == ORACLE_MODE_ADMM) ? 4 * H - 1 : H;
    const long long total = cols ? ncols : (long long)N * J;
    if (nthreads < 1) nthreads = 1;
    int err = 0;
#pragma omp parallel num_threads(nthreads)
    {
        double *work = malloc(sizeof(double) * 6 * 8 * (size_t)H + 64);
        double *xc = malloc(sizeof(double) * H), *xic = malloc(sizeof(double) * H);
        double *xin = malloc(sizeof(double) * H), *dc = malloc(sizeof(double) * D);
        double *din = malloc(sizeof(double) * D);
        double bnd[8];
        if (!work || !xc || !xic || !xin || !dc || !din) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (long long t = 0; t < total; ++t) {
                long long c = cols ? cols[t] : t;
                if (c < 0 || c >= (long long)N * J) continue;
                long long nn = c / J;
                int j = (int)(c % J);
                for (int b = 0; b < 8; ++b) bnd[b] = bounds[b * J + j];
                for (int i = 0; i < H; ++i) xic[i] = xi[(nn * H + i) * J + j];
                if (x_init)
                    for (int i = 0; i < H; ++i) xin[i] = x_init[(nn * H + i) * J + j];
                if (dual_init)
                    for (int i = 0; i < D; ++i) din[i] = dual_init[(nn * D + i) * J + j];
                double pr, du;
                solve_column(&S, bnd, q0[j], v0[j], xic, iters, x_init ? xin : NULL,
                             dual_init ? din : NULL, xc, dc, &pr, &du, work);
                for (int i = 0; i < H; ++i) x_out[(nn * H + i) * J + j] = xc[i];
                if (primal) primal[nn * J + j] = pr;
                if (dual) dual[nn * J + j] = du;
                if (dual_out)
                    for (int i = 0; i < D; ++i) dual_out[(nn * D + i) * J + j] = dc[i];
            }
        }
        free(work); free(xc); free(xic); free(xin); free(dc); free(din);
    }
    setup_free(&S);
    return err;
}

/* ---------------------------------------------------------------------------
 * The exact projection Pi(xi) of one column (Sec. III-C: the minimal-l2
 * projection onto the feasible set), obtained by running the ADMM iteration
 * with row scaling and rho = 1 until the last primal step is below tol_step
 * and the row-normalised violation below tol_viol, or max_iters.  Returns the
 * number of iterations used (negative on error).  x_out has H entries.
 * ------------------------------------------------------------------------- */
long long oracle_exact_projection(int H, double dt, const double *bnd, double q0, double v0,
                                  const double *xi, double tol_step, double tol_viol,
                                  long long max_iters, double *x_out, double *viol_out)
{
    setup_t S;
    if (setup_make(&S, ORACLE_MODE_ADMM, ORACLE_SCALE_ROWNORM, H, dt, 1.0) != 0) return -1;
    const int p = S.p;
    double *work = malloc(sizeof(double) * 6 * 8 * (size_t)H + 64);
    double *u = calloc((size_t)p, sizeof(double));
    double *x = malloc(sizeof(double) * H);
    if (!work || !u || !x) { free(work); free(u); free(x); setup_free(&S); return -2; }
    long long it = 0;
    double pr = 0.0, du = 0.0;
    const int chunk = 50;
    solve_column(&S, bnd, q0, v0, xi, chunk, NULL, NULL, x, u, &pr, &du, work);
    it = chunk;
    while ((du > tol_step || pr > tol_viol) && it < max_iters) {
        double *xw = malloc(sizeof(double) * H), *uw = malloc(sizeof(double) * p);
        memcpy(xw, x, sizeof(double) * H);
        memcpy(uw, u, sizeof(double) * p);
        solve_column(&S, bnd, q0, v0, xi, chunk, xw, uw, x, u, &pr, &du, work);
        free(xw); free(uw);
        it += chunk;
    }
    memcpy(x_out, x, sizeof(double) * H);
    if (viol_out) *viol_out = pr;
    free(work); free(u); free(x);
    setup_free(&S);
    return it;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Sampling of Alg. 1 ("Draw a batch of n velocity-sequence samples from
 * N(nu, Sigma)", diagonal Sigma): xi[n][k][j] = mean[k][j] + std[k][j] * z with
 * z standard normal.  The normals come from the counter-based generator
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011) and the Box-Muller transform, so that any element can
 * be drawn independently:
 *   element e = (n*H + k)*J + j;  block q = e / 4;  counter = (q_lo, q_hi,
 *   stream_lo, stream_hi), key = (seed_lo, seed_hi);  the block's four words
 *   w0..w3 give u = (w + 0.5) / 2^32 and the pairs (w0,w1), (w2,w3) give
 *   z = sqrt(-2 ln u_a) * (cos(2 pi u_b), sin(2 pi u_b)); element e takes
 *   output e % 4 of its block.
 * ------------------------------------------------------------------------- */
static void philox_round(unsigned int c[4], const unsigned int k[2])
{
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c[0];
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c[2];
    const unsigned int hi0 = (unsigned int)(p0 >> 32), lo0 = (unsigned int)p0;
    const unsigned int hi1 = (unsigned int)(p1 >> 32), lo1 = (unsigned int)p1;
    const unsigned int n0 = hi1 ^ c[1] ^ k[0];
    const unsigned int n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const unsigned int ctr_in[4], const unsigned int key_in[2], unsigned int out[4])
{
    unsigned int c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    unsigned int k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

int oracle_sample_batch(int N, int H, int J, const double *mean, const double *stdv,
                        unsigned long long seed, unsigned long long stream, double *xi)
{
    if (N < 0 || H < 1 || J < 1) return -1;
    const long long total = (long long)N * H * J;
    const unsigned int key[2] = {(unsigned int)seed, (unsigned int)(seed >> 32)};
    const double two_pi = 6.283185307179586476925286766559;
    for (long long q = 0; q * 4 < total; ++q) {
        const unsigned int ctr[4] = {(unsigned int)q, (unsigned int)((unsigned long long)q >> 32),
                                     (unsigned int)stream, (unsigned int)(stream >> 32)};
        unsigned int w[4];
        oracle_philox4x32_10(ctr, key, w);
        double u[4], z[4];
        for (int i = 0; i < 4; ++i) u[i] = ((double)w[i] + 0.5) * (1.0 / 4294967296.0);
        for (int p = 0; p < 2; ++p) {
            const double r = sqrt(-2.0 * log(u[2 * p]));
            z[2 * p] = r * cos(two_pi * u[2 * p + 1]);
            z[2 * p + 1] = r * sin(two_pi * u[2 * p + 1]);
        }
        for (int i = 0; i < 4; ++i) {
            const long long e = q * 4 + i;
            if (e >= total) break;
            const long long kj = e % ((long long)H * J);
            xi[e] = mean[kj] + stdv[kj] * z[i];
        }
    }
    return 0;
}
