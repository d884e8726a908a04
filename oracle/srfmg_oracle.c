/*
 * srfmg_oracle.c -- plain, serial, FP64 CPU oracle for the one-pass FMG-FAS
 * solve with segmental refinement (SR) of
 *   M. F. Adams, "A low memory, highly concurrent multigrid algorithm".
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct restatement
 * of the method that the CUDA path is checked against.  Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Problem (Sec. 4): -u'' = f on (0,1), u(0) = u(1) = 0, cell-centred second
 * order finite volumes.  Also the nonlinear problem -u'' + lam e^u = f (the
 * Bratu equation, lam >= 0) with the same discretisation, solved by the same
 * FAS cycles (Sec. 2.2, Eqs. 1-2: the coarse equation of a nonlinear operator;
 * Fig. 1: a nonlinear smoother S(L, u, f)); the paper's studies are linear,
 * so the nonlinear pieces carry "Reading:" notes.  And -(a u')' = f with a
 * coefficient a > 0 given at the cell faces of the finest level (the paper's
 * studies have a = 1): fluxes F_{i+1/2} = a_{i+1/2} (u_{i+1} - u_i), the same
 * cycles; "Reading:" notes mark its pieces.  Level l has n = 2^l cells of width h = 1/n, centres
 * x_i = (i + 1/2) h; the Dirichlet wall is an odd ghost cell (u_{-1} = -u_0,
 * u_n = -u_{n-1}), which is where the diagonal 3/h^2 of the first and last
 * rows of the appendix operator comes from.
 *
 * Arithmetic: IEEE double, built with -ffp-contract=off.  The operator is
 * applied in flux form, (L u)_i = (F_{i-1/2} - F_{i+1/2}) / h^2 with
 * F_{i+1/2} = u_{i+1} - u_i; the difference of two nearby doubles is exact,
 * so residuals carry no O(eps |u| / h^2) rounding noise.
 *
 * The routines follow the paper's algorithms in its order:
 *   Fig. 1 (FAS V-cycle), Fig. 2 (FMG), Eq. 4 (correction update), Eq. 5
 *   (full update), Eqs. 6-7 (tau correction), Fig. 3 (FMG-FAS-SR), Fig. 5
 *   (Kaczmarz compatible relaxation) and the operators of Sec. 4.
 * Points where the paper is silent carry a "Reading:" note.
 *
 * Vectors are passed as (array, offset) pairs: a[i - off] holds cell i.  The
 * stored levels use offset 0; a segment's patch buffer uses the index of its
 * first cell.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXLEV 31

/* Parameters of one solve.  Level tables are indexed by level l. */
typedef struct {
    int32_t M;              /* finest level, N = 2^M cells */
    int32_t M0;             /* coarsest level (exact solve), >= 2 */
    int32_t nRS;            /* number of SR levels: {M-nRS+1 .. M} */
    int32_t nu1, nu2;       /* V(nu1, nu2) */
    int32_t smoother;       /* 0: lexicographic Gauss-Seidel, direction reversed
                                  after every sweep (appendix; default);
                               1: red-black Gauss-Seidel, even cells first */
    int32_t tau_src;        /* 0: tau from the assembled level, as the appendix
                                  program computes it (default);
                               1: tau from each segment's own extended patch,
                                  the literal reading of Fig. 3 line 4 */
    int32_t seg_w[OR_MAXLEV + 1]; /* per level: segment interior width, 0 = whole level */
    int32_t seg_b[OR_MAXLEV + 1]; /* per level: buffer cells on each side */
    int32_t op;             /* 0: -u'' = f;  1: -u'' + lam e^u = f;  2: -(a u')' = f */
    double lam;             /* op 1: lam >= 0 (op 0: ignored) */
    const double *coef;     /* op 2: a at the 2^coef_level + 1 faces x = j 2^-coef_level */
    int32_t coef_level;     /* op 2: the level coef is given on (the finest) */
    int32_t post;           /* post-smoothing leg of an SR level: 0: the full update
                                  u_l = Pi u_{l-1} (Eq. 5) with compatible relaxation
                                  (Fig. 5), the paper's (default); 1: the FAS
                                  correction (Eq. 4) of the pre-smoothed level, which
                                  the serial SR variant recomputes segment by segment,
                                  then S without Kaczmarz */
} or_params;

/* lam of the operator (0 for the linear problem). */
static double op_lam(const or_params *p) { return p->op == 1 ? p->lam : 0.0; }

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

static double cell(const double *a, int off, int i) { return a[i - off]; }

/* ------------------------------------------------------------------ */
/* Operators of Sec. 4 (one level of n cells, h = 1/n)                 */
/* ------------------------------------------------------------------ */

/* Face coefficient a_j of a level (faces x = j h, j = 0..n); a = NULL is the
 * constant coefficient 1 (every product with it is then exact, so the
 * constant-coefficient results are unchanged bit for bit). */
static double coef(const double *a, int j) { return a ? a[j] : 1.0; }

/* F_{i-1/2} = a_i (u_i - u_{i-1}); at the left wall F_{-1/2} = a_0 (u_0 - (-u_0)). */
static double flux_left(const double *u, int off, int i, const double *a) {
    return coef(a, i) * (i == 0 ? 2.0 * cell(u, off, 0) : cell(u, off, i) - cell(u, off, i - 1));
}
/* F_{i+1/2} = a_{i+1} (u_{i+1} - u_i); at the right wall F_{n-1/2} = a_n ((-u_{n-1}) - u_{n-1}). */
static double flux_right(const double *u, int off, int i, int n, const double *a) {
    return coef(a, i + 1) * (i == n - 1 ? -2.0 * cell(u, off, n - 1) : cell(u, off, i + 1) - cell(u, off, i));
}
/* (L u)_i = (F_{i-1/2} - F_{i+1/2}) / h^2, with 1/h^2 = n^2 exactly. */
static double Lu_at(const double *u, int off, int i, int n, const double *a) {
    double inv_h2 = (double)n * (double)n;
    return (flux_left(u, off, i, a) - flux_right(u, off, i, n, a)) * inv_h2;
}
/* Diagonal of L: (a_i + a_{i+1}) / h^2, with 2 a at a wall face (2/h^2 inside
 * and 3/h^2 in the two wall cells for a = 1). */
static double Ldiag_at(int i, int n, const double *a) {
    double inv_h2 = (double)n * (double)n;
    double al = coef(a, i) * (i == 0 ? 2.0 : 1.0), ar = coef(a, i + 1) * (i == n - 1 ? 2.0 : 1.0);
    return (al + ar) * inv_h2;
}

/* Nonlinear operator N(u)_i = (L u)_i + lam e^{u_i}.  With lam = 0 the added
 * term is an exact +0, so N is L bit for bit. */
static double Nu_at(const double *u, int off, int i, int n, double lam, const double *a) {
    return Lu_at(u, off, i, n, a) + lam * exp(cell(u, off, i));
}

/* Restriction (Sec. 4, first order): mean of the two children of coarse J. */
static double restrict_at(const double *uf, int off, int J) {
    return (cell(uf, off, 2 * J) + cell(uf, off, 2 * J + 1)) * 0.5;
}

/* Coarse value with the odd reflection at the walls (both prolongations). */
static double coarse_ghost(const double *uc, int j, int nc) {
    if (j < 0) return -uc[-j - 1];
    if (j >= nc) return -uc[2 * nc - 1 - j];
    return uc[j];
}

/* Second order prolongation P (Sec. 4): a child takes 3/4 of its parent and
 * 1/4 of the parent's neighbour on its side; odd reflection at a wall. */
static double prolong_lin_at(const double *uc, int i, int nc) {
    int J = i >> 1;
    int nb = (i & 1) ? J + 1 : J - 1;
    return (3.0 * uc[J] + coarse_ghost(uc, nb, nc)) * 0.25;
}

/* Fourth order FMG interpolation Pi (Sec. 4): cubic Lagrange interpolation
 * at the child centre (1/4 of a coarse cell left or right of its parent)
 * through the four nearest coarse centres: weights (-5, 35, 105, -7)/128 for
 * the left child and the mirror for the right child.  The appendix's special
 * rows at the walls are this formula with odd ghosts. */
static double prolong_fmg_at(const double *uc, int i, int nc) {
    int J = i >> 1;
    double s;
    if ((i & 1) == 0)
        s = -5.0 * coarse_ghost(uc, J - 2, nc) + 35.0 * coarse_ghost(uc, J - 1, nc)
            + 105.0 * uc[J] - 7.0 * coarse_ghost(uc, J + 1, nc);
    else
        s = -7.0 * coarse_ghost(uc, J - 1, nc) + 105.0 * uc[J]
            + 35.0 * coarse_ghost(uc, J + 1, nc) - 5.0 * coarse_ghost(uc, J + 2, nc);
    return s / 128.0;
}

/* Exact solve of L u = rhs on one level (the coarsest-grid solve of Figs. 1-2):
 * L is tridiagonal and diagonally dominant, so the Thomas algorithm. */
static int thomas_shift(int n, const double *rhs, const double *dshift, double *u, const double *a);
static int thomas(int n, const double *rhs, double *u) { return thomas_shift(n, rhs, NULL, u, NULL); }

/* Thomas for the tridiagonal L + diag(dshift) (dshift = NULL: L); the
 * coefficient a of the level (NULL: 1). */
static int thomas_shift(int n, const double *rhs, const double *dshift, double *u, const double *a) {
    if (n < 1) return OR_EINVAL;
    double *cp = (double *)calloc((size_t)n, sizeof(double));
    double *dp = (double *)calloc((size_t)n, sizeof(double));
    if (!cp || !dp) { free(cp); free(dp); return OR_ENOMEM; }
    double off = -((double)n * (double)n);
    for (int i = 0; i < n; i++) {
        double lower = i > 0 ? coef(a, i) * off : 0.0;
        double upper = i < n - 1 ? coef(a, i + 1) * off : 0.0;
        double diag = dshift ? Ldiag_at(i, n, a) + dshift[i] : Ldiag_at(i, n, a);
        double denom = diag - (i > 0 ? lower * cp[i - 1] : 0.0);
        cp[i] = upper / denom;
        dp[i] = (rhs[i] - (i > 0 ? lower * dp[i - 1] : 0.0)) / denom;
    }
    u[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) u[i] = dp[i] - cp[i] * u[i + 1];
    free(cp); free(dp);
    return OR_OK;
}

/* Exact solve of N(u) = rhs on the coarsest level (Figs. 1-2: "exact solve of
 * coarsest grid").  Linear: Thomas.  Reading (nonlinear): Newton's method from
 * the iterate passed in u (the restricted FAS iterate; zero in the first FMG
 * step), each step a Thomas solve with the Jacobian L + diag(lam e^u), until
 * the step is at most 4 ulp of max|u| or stops shrinking (the unique solution
 * for lam >= 0 to rounding; at most 100 steps). */
static int coarsest_solve(const or_params *p, int n, const double *rhs, double *u, const double *a) {
    double lam = op_lam(p);
    if (lam == 0.0) return thomas_shift(n, rhs, NULL, u, a);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *du = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = (r && d && du) ? OR_OK : OR_ENOMEM;
    double prev = INFINITY;
    for (int it = 0; it < 100 && rc == OR_OK; it++) {
        for (int i = 0; i < n; i++) {
            r[i] = rhs[i] - Nu_at(u, 0, i, n, lam, a);
            d[i] = lam * exp(u[i]);
        }
        rc = thomas_shift(n, r, d, du, a);
        if (rc) break;
        double step = 0.0, umax = 0.0;
        for (int i = 0; i < n; i++) {
            u[i] += du[i];
            step = fmax(step, fabs(du[i]));
            umax = fmax(umax, fabs(u[i]));
        }
        if (step <= 4.0 * DBL_EPSILON * umax || step >= prev) break;
        prev = step;
    }
    free(r); free(d); free(du);
    return rc;
}

/* ------------------------------------------------------------------ */
/* The smoother S of Sec. 3 and Fig. 5 on one extended patch           */
/* ------------------------------------------------------------------ */

/* One Gauss-Seidel update (omega = 1): u_i += (f_i - (L u)_i) / L_ii.
 * Reading (nonlinear, the smoother S(L, u, f) of Fig. 1): one pointwise Newton
 * step, u_i += (f_i - N(u)_i) / (L_ii + lam e^{u_i}); with lam = 0 both added
 * terms are exact zeros and this is the linear update bit for bit. */
static void gs_update(double *v, int voff, const double *rhs, int roff, int i, int n, double lam,
                      const double *a) {
    double e = lam * exp(cell(v, voff, i));
    v[i - voff] = cell(v, voff, i) + (cell(rhs, roff, i) - (Lu_at(v, voff, i, n, a) + e)) / (Ldiag_at(i, n, a) + e);
}

/* Kaczmarz pass of Fig. 5 over every coarse cell J whose children both lie in
 * [e0, e1): r = uH_J - (R v)_J, t = r / (R R^T)_JJ = r / (1/2), and
 * v += R(J,:)^T t, i.e. each child gets t/2.  The pairs are disjoint, so the
 * order of J does not matter.  Reading: e0 is even (segments and buffers have
 * even widths), so the pairs are the true sibling pairs. */
static void kaczmarz_pass(double *v, int voff, const double *uH, int e0, int e1) {
    for (int i = e0; i + 1 < e1; i += 2) {
        int J = i >> 1;
        double r = uH[J] - restrict_at(v, voff, J);
        double t = r / 0.5;
        v[i - voff] = cell(v, voff, i) + 0.5 * t;
        v[i + 1 - voff] = cell(v, voff, i + 1) + 0.5 * t;
    }
}

/* nsweeps iterations of S on the cells [e0, e1); v also holds the frozen cells
 * just outside [e0, e1) (read, never written).  With uH != NULL every
 * iteration starts with the Kaczmarz pass (compatible relaxation, Fig. 5,
 * whose order "Kaczmarz, then the standard smoother" the appendix keeps).
 * Then one Gauss-Seidel sweep:
 *   smoother 0: lexicographic, ascending first and reversed after every
 *     sweep of the call (the appendix's "symmetrize");
 *   smoother 1: every even cell of [e0,e1), then every odd cell (red-black;
 *     colour = global cell index mod 2).  Kept as an option: with V(1,1) on
 *     this discretization its V-cycle factor grows with the depth and one FMG
 *     cycle misses discretization accuracy. */
static void patch_sweeps(int smoother, double *v, int voff, const double *rhs, int roff,
                         int n, int e0, int e1, int nsweeps, const double *uH, double lam, const double *a) {
    int ascending = 1;
    for (int k = 0; k < nsweeps; k++) {
        if (uH) kaczmarz_pass(v, voff, uH, e0, e1);
        if (smoother == 1) {
            for (int colour = 0; colour < 2; colour++)
                for (int i = e0; i < e1; i++)
                    if ((i & 1) == colour) gs_update(v, voff, rhs, roff, i, n, lam, a);
        } else {
            if (ascending) for (int i = e0; i < e1; i++) gs_update(v, voff, rhs, roff, i, n, lam, a);
            else           for (int i = e1 - 1; i >= e0; i--) gs_update(v, voff, rhs, roff, i, n, lam, a);
            ascending = !ascending;
        }
    }
}

/* Extended patch of the segment with interior [s, s+w) on a level of n cells:
 * E = [s - b, s + w + b) clipped to the domain (Sec. 3, buffer cells), and
 * the cells [lo, hi) the patch reads: E plus one frozen cell on each side
 * that lies inside the domain. */
static void extended_patch(int s, int w, int b, int n, int *e0, int *e1, int *lo, int *hi) {
    *e0 = s - b < 0 ? 0 : s - b;
    *e1 = s + w + b > n ? n : s + w + b;
    *lo = *e0 > 0 ? *e0 - 1 : 0;
    *hi = *e1 < n ? *e1 + 1 : n;
}

/* ------------------------------------------------------------------ */
/* tau-corrected coarse right-hand side (Eqs. 6-7, Fig. 3 lines 3-5)   */
/* ------------------------------------------------------------------ */

/* rhs_c(J) = (R rhs_f)_J + (L_c R ubar)_J - (R L_f ubar)_J, evaluated left to
 * right as in the appendix's down leg.  The restricted solution R ubar plays
 * the role of Ihat ubar in Eq. 7 (Ihat = I here).  Reads fine cells 2J-2 ..
 * 2J+3 of ubar (fewer at a wall) and 2J, 2J+1 of rhs_f. */
static double tau_rhs_at(const double *ubar, int uoff, const double *rhs_f, int roff,
                         int J, int nf, double lam, const double *af, const double *ac) {
    int nc = nf / 2;
    double Rrhs = (cell(rhs_f, roff, 2 * J) + cell(rhs_f, roff, 2 * J + 1)) * 0.5;
    double inv_H2 = (double)nc * (double)nc;
    double uJ = restrict_at(ubar, uoff, J);
    /* Reading (variable coefficient): the coarse operator has the coefficients
     * of the coinciding fine faces (coarse face J is fine face 2J) */
    double Gl = coef(ac, J) * (J == 0 ? 2.0 * uJ : uJ - restrict_at(ubar, uoff, J - 1));
    double Gr = coef(ac, J + 1) * (J == nc - 1 ? -2.0 * uJ : restrict_at(ubar, uoff, J + 1) - uJ);
    /* nonlinear (Eq. 2 with N for L): N_c(R ubar) - R N_f(ubar); lam = 0 adds
     * exact zeros */
    double Lc = (Gl - Gr) * inv_H2 + lam * exp(uJ);
    double RLf = (Nu_at(ubar, uoff, 2 * J, nf, lam, af) + Nu_at(ubar, uoff, 2 * J + 1, nf, lam, af)) * 0.5;
    return (Rrhs + Lc) - RLf;
}

/* ------------------------------------------------------------------ */
/* Every level stored ("horizontal" processing, Sec. 4)                */
/* ------------------------------------------------------------------ */

typedef struct {
    const or_params *p;
    double *u[OR_MAXLEV + 1];
    double *rhs[OR_MAXLEV + 1];
    double *tmp;      /* scratch, 2^M doubles */
    double *tmp2;     /* scratch, 2^M doubles */
    double *patch;    /* one extended patch incl. frozen cells */
    double *a[OR_MAXLEV + 1];   /* op 2: face coefficients of each level, else NULL */
} or_state;

/* Face coefficients of level l (2^l + 1 values) for op 2, else NULL.
 * Reading (variable coefficient): every face of level l coincides with a face
 * of the finest level, whose coefficient it takes (injection). */
static double *level_coef(const or_params *p, int l) {
    if (p->op != 2) return NULL;
    int n = 1 << l, sh = p->coef_level - l;
    double *a = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (a)
        for (int j = 0; j <= n; j++) a[j] = p->coef[(size_t)j << sh];
    return a;
}

static int is_sr_level(const or_params *p, int l) { return l > p->M - p->nRS; }
static int segmented(const or_params *p, int l) {
    return p->seg_w[l] != 0 && p->seg_w[l] < (1 << l);
}

/* S applied to a whole level (Sec. 3): a level that is not segmented is one
 * patch; otherwise each segment's extended patch is smoothed from a copy of
 * the input and only its interior is kept, i.e. the patch solves are
 * assembled additively (block Jacobi), independent of processing order. */
static void smooth_level(or_state *st, int l, const double *u_in, double *u_out,
                         int nsweeps, const double *uH) {
    const or_params *p = st->p;
    int n = 1 << l;
    if (!segmented(p, l)) {
        if (u_out != u_in) memcpy(u_out, u_in, sizeof(double) * (size_t)n);
        patch_sweeps(p->smoother, u_out, 0, st->rhs[l], 0, n, 0, n, nsweeps, uH, op_lam(p), st->a[l]);
        return;
    }
    int w = p->seg_w[l];
    for (int s = 0; s < n; s += w) {
        int e0, e1, lo, hi;
        extended_patch(s, w, p->seg_b[l], n, &e0, &e1, &lo, &hi);
        memcpy(st->patch, u_in + lo, sizeof(double) * (size_t)(hi - lo));
        patch_sweeps(p->smoother, st->patch, lo, st->rhs[l], 0, n, e0, e1, nsweeps, uH, op_lam(p), st->a[l]);
        memcpy(u_out + s, st->patch + (s - lo), sizeof(double) * (size_t)w);
    }
}

/* Pre-smoothing of level l and the transfer to level l-1 (Fig. 3 lines 2-5,
 * appendix down leg): u_l <- S(u_l); u_{l-1} <- R u_l;
 * rhs_{l-1} <- R rhs_l + L_{l-1} R u_l - R L_l u_l.
 * Reading (tau_src = 0, default): both come from the assembled level, as in
 * the appendix program, which the paper states has the same semantics as
 * Fig. 3.  With tau_src = 1 each segment forms them on its interior coarse
 * cells from its own smoothed extended patch ubar (Fig. 3 line 4 read
 * literally); tau at a segment edge then reads buffer cells that differ from
 * the assembled values the restricted solution comes from. */
static void presmooth_and_restrict(or_state *st, int l) {
    const or_params *p = st->p;
    int n = 1 << l, nc = n / 2;
    double *ul = st->u[l], *uc = st->u[l - 1], *rc = st->rhs[l - 1], *rf = st->rhs[l];
    if (!segmented(p, l) || p->tau_src == 0) {
        smooth_level(st, l, ul, st->tmp, p->nu1, NULL);
        memcpy(ul, st->tmp, sizeof(double) * (size_t)n);
        for (int J = 0; J < nc; J++) uc[J] = restrict_at(ul, 0, J);
        for (int J = 0; J < nc; J++) rc[J] = tau_rhs_at(ul, 0, rf, 0, J, n, op_lam(p), st->a[l], st->a[l - 1]);
        return;
    }
    int w = p->seg_w[l];
    for (int s = 0; s < n; s += w) {
        int e0, e1, lo, hi;
        extended_patch(s, w, p->seg_b[l], n, &e0, &e1, &lo, &hi);
        memcpy(st->patch, ul + lo, sizeof(double) * (size_t)(hi - lo));
        patch_sweeps(p->smoother, st->patch, lo, rf, 0, n, e0, e1, p->nu1, NULL, op_lam(p), st->a[l]);
        memcpy(st->tmp + s, st->patch + (s - lo), sizeof(double) * (size_t)w);
        for (int J = s / 2; J < (s + w) / 2; J++) {
            uc[J] = restrict_at(st->patch, lo, J);
            rc[J] = tau_rhs_at(st->patch, lo, rf, 0, J, n, op_lam(p), st->a[l], st->a[l - 1]);
        }
    }
    memcpy(ul, st->tmp, sizeof(double) * (size_t)n);
}

/* Post-smoothing leg update of level l from the corrected level l-1
 * (Fig. 3 post-smoothing leg, appendix up leg):
 *   SR level:  u_l <- Pi u_{l-1} (Eq. 5, full update), then S with the
 *              Kaczmarz compatible relaxation against u_{l-1} (Fig. 5);
 *   otherwise: u_l <- u_l + P (u_{l-1} - R u_l) (Eq. 4), then S. */
static void postsmooth_update(or_state *st, int l) {
    const or_params *p = st->p;
    int n = 1 << l, nc = n / 2;
    double *ul = st->u[l], *uc = st->u[l - 1], *t = st->tmp;
    if (is_sr_level(p, l) && p->post == 0) {
        for (int i = 0; i < n; i++) t[i] = prolong_fmg_at(uc, i, nc);
        smooth_level(st, l, t, ul, p->nu2, uc);
    } else {
        double *corr = st->tmp2;
        for (int J = 0; J < nc; J++) corr[J] = uc[J] - restrict_at(ul, 0, J);
        for (int i = 0; i < n; i++) t[i] = ul[i] + prolong_lin_at(corr, i, nc);
        smooth_level(st, l, t, ul, p->nu2, NULL);
    }
}

/* One FAS V-cycle (Fig. 1) with finest level `top`; u[top], rhs[top] set.
 * Each level is smoothed and transferred down, the coarsest level M0 is
 * solved exactly, and each level is corrected and smoothed on the way up. */
static int vcycle(or_state *st, int top) {
    const or_params *p = st->p;
    for (int l = top; l > p->M0; l--) presmooth_and_restrict(st, l);
    int rc = coarsest_solve(p, 1 << p->M0, st->rhs[p->M0], st->u[p->M0], st->a[p->M0]);
    if (rc) return rc;
    for (int l = p->M0 + 1; l <= top; l++) postsmooth_update(st, l);
    return OR_OK;
}

static void free_state(or_state *st) {
    for (int l = 0; l <= OR_MAXLEV; l++) { free(st->u[l]); free(st->rhs[l]); free(st->a[l]); }
    free(st->tmp); free(st->tmp2); free(st->patch);
}

static int check_params(const or_params *p) {
    if (p->M0 < 2 || p->M < p->M0 || p->M > 28) return OR_EINVAL;
    if (p->nRS < 0 || p->nRS > p->M - p->M0) return OR_EINVAL;
    if (p->op != 0 && p->op != 1 && p->op != 2) return OR_EINVAL;
    if (p->op == 1 && !(p->lam >= 0.0 && p->lam < INFINITY)) return OR_EINVAL;
    if (p->op == 2) {
        if (!p->coef || p->coef_level < p->M || p->coef_level > 28) return OR_EINVAL;
        for (long long j = 0; j <= (1LL << p->coef_level); j++)
            if (!(p->coef[j] > 0.0 && p->coef[j] < INFINITY)) return OR_EINVAL;
    }
    if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 > 16 || p->nu2 > 16) return OR_EINVAL;
    if (p->smoother < 0 || p->smoother > 1 || p->tau_src < 0 || p->tau_src > 1) return OR_EINVAL;
    if (p->post < 0 || p->post > 1) return OR_EINVAL;
    for (int l = p->M0 + 1; l <= p->M; l++) {
        int w = p->seg_w[l], b = p->seg_b[l], n = 1 << l;
        if (w == 0) continue;
        if (w < 2 || (w & (w - 1)) || w > n) return OR_EINVAL;
        if (w < n && (b < 2 || (b & 1) || b > (1 << 20))) return OR_EINVAL;
    }
    return OR_OK;
}

static int max_patch(const or_params *p) {
    int m = 4;
    for (int l = p->M0 + 1; l <= p->M; l++)
        if (p->seg_w[l] && p->seg_w[l] + 2 * p->seg_b[l] + 2 > m) m = p->seg_w[l] + 2 * p->seg_b[l] + 2;
    return m;
}

static int alloc_state(or_state *st, const or_params *p) {
    memset(st, 0, sizeof(*st));
    st->p = p;
    for (int l = p->M0; l <= p->M; l++) {
        st->u[l] = (double *)calloc((size_t)1 << l, sizeof(double));
        st->rhs[l] = (double *)calloc((size_t)1 << l, sizeof(double));
        st->a[l] = level_coef(p, l);
        if (!st->u[l] || !st->rhs[l] || (p->op == 2 && !st->a[l])) { free_state(st); return OR_ENOMEM; }
    }
    st->tmp = (double *)calloc((size_t)1 << p->M, sizeof(double));
    st->tmp2 = (double *)calloc((size_t)1 << p->M, sizeof(double));
    st->patch = (double *)calloc((size_t)max_patch(p), sizeof(double));
    if (!st->tmp || !st->tmp2 || !st->patch) { free_state(st); return OR_ENOMEM; }
    return OR_OK;
}

/* Right-hand sides on every level (appendix operator set-up): rhs_M = f and
 * each coarser level is the restriction of the next finer one. */
static void rhs_hierarchy(or_state *st, int top, const double *f_top) {
    const or_params *p = st->p;
    memcpy(st->rhs[top], f_top, sizeof(double) * ((size_t)1 << top));
    for (int l = top; l > p->M0; l--)
        for (int J = 0; J < (1 << (l - 1)); J++) st->rhs[l - 1][J] = restrict_at(st->rhs[l], 0, J);
}

/* FMG (Fig. 2) up to level `top`: exact solve on M0, then for each finer level
 * the FMG interpolation Pi followed by one V-cycle. */
static int fmg_up_to(or_state *st, int top) {
    const or_params *p = st->p;
    int rc = coarsest_solve(p, 1 << p->M0, st->rhs[p->M0], st->u[p->M0], st->a[p->M0]);
    for (int k = p->M0; k < top && !rc; k++) {
        int nc = 1 << k;
        for (int i = 0; i < 2 * nc; i++) st->u[k + 1][i] = prolong_fmg_at(st->u[k], i, nc);
        rc = vcycle(st, k + 1);
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Exported entry points                                               */
/* ------------------------------------------------------------------ */

int or_apply_L(int n, const double *u, double *out) {
    for (int i = 0; i < n; i++) out[i] = Lu_at(u, 0, i, n, NULL);
    return OR_OK;
}
int or_restrict(int nc, const double *uf, double *uc) {
    for (int J = 0; J < nc; J++) uc[J] = restrict_at(uf, 0, J);
    return OR_OK;
}
int or_prolong_lin(int nc, const double *uc, double *uf) {
    for (int i = 0; i < 2 * nc; i++) uf[i] = prolong_lin_at(uc, i, nc);
    return OR_OK;
}
int or_prolong_fmg(int nc, const double *uc, double *uf) {
    if (nc < 2) return OR_EINVAL;
    for (int i = 0; i < 2 * nc; i++) uf[i] = prolong_fmg_at(uc, i, nc);
    return OR_OK;
}
int or_thomas(int n, const double *rhs, double *u) { return thomas(n, rhs, u); }

/* tau-corrected coarse rhs from an assembled fine vector, every coarse cell. */
int or_tau_rhs(int nf, const double *ubar, const double *rhs_f, double *rhs_c) {
    for (int J = 0; J < nf / 2; J++) rhs_c[J] = tau_rhs_at(ubar, 0, rhs_f, 0, J, nf, 0.0, NULL, NULL);
    return OR_OK;
}

/* The nonlinear operator N(u) = L u + lam e^u on one level of n cells. */
int or_apply_N(int n, double lam, const double *u, double *out) {
    for (int i = 0; i < n; i++) out[i] = Nu_at(u, 0, i, n, lam, NULL);
    return OR_OK;
}

/* The variable-coefficient operator -(a u')' on one level of n cells with the
 * face coefficients a[0..n]. */
int or_apply_La(int n, const double *a, const double *u, double *out) {
    for (int i = 0; i < n; i++) out[i] = Lu_at(u, 0, i, n, a);
    return OR_OK;
}

/* Gradient of a loss L through the solution of A(a) u = f with respect to the
 * logarithm of the face coefficients, by the adjoint state (the paper has no
 * gradient; this is the derivative of the variable-coefficient operator of the
 * Sec. 4 discretisation).  lam = A^{-T} dL/du = A^{-1} dL/du (A is symmetric).
 * Face f (between cells f-1 and f) carries the flux a_f (u_f - u_{f-1}) n^2,
 * which enters (A u)_f with + and (A u)_{f-1} with -, so
 *   dL/da_f = -lam^T (dA/da_f) u = -(u_f - u_{f-1}) (lam_f - lam_{f-1}) n^2;
 * the wall faces enter one cell only, through the odd ghost: 2 a_0 u_0 n^2 in
 * (A u)_0 and 2 a_n u_{n-1} n^2 in (A u)_{n-1}.  out[f] = a_f dL/da_f, f = 0..n. */
int or_coef_gradient(int n, const double *a, const double *u, const double *lam, double *out) {
    if (n < 1) return OR_EINVAL;
    const double n2 = (double)n * (double)n;
    out[0] = -(a[0] * (2.0 * u[0]) * lam[0]) * n2;
    for (int f = 1; f < n; f++) out[f] = -(a[f] * (u[f] - u[f - 1]) * (lam[f] - lam[f - 1])) * n2;
    out[n] = -(a[n] * (2.0 * u[n - 1]) * lam[n - 1]) * n2;
    return OR_OK;
}

/* The coarsest-level solve of p on n cells: rhs in, u = starting iterate in,
 * solution out. */
int or_coarsest(const or_params *p, int n, const double *rhs, double *u) {
    if (p->op != 0 && p->op != 1 && p->op != 2) return OR_EINVAL;
    int l = 0;
    while ((1 << l) < n) l++;
    if ((1 << l) != n || (p->op == 2 && (!p->coef || p->coef_level < l))) return OR_EINVAL;
    double *a = level_coef(p, l);
    if (p->op == 2 && !a) return OR_ENOMEM;
    int rc = coarsest_solve(p, n, rhs, u, a);
    free(a);
    return rc;
}

/* One application of the level smoother S (segmentation from p->seg_w[l]). */
int or_smooth(const or_params *p, int l, const double *u_in, const double *rhs,
              int nsweeps, const double *uH, double *u_out) {
    if (check_params(p) || l < 1 || l > OR_MAXLEV) return OR_EINVAL;
    or_state st;
    memset(&st, 0, sizeof(st));
    st.p = p;
    st.rhs[l] = (double *)rhs;
    st.patch = (double *)calloc((size_t)max_patch(p), sizeof(double));
    st.a[l] = level_coef(p, l);
    if (!st.patch || (p->op == 2 && !st.a[l])) { free(st.patch); free(st.a[l]); return OR_ENOMEM; }
    smooth_level(&st, l, u_in, u_out, nsweeps, uH);
    free(st.patch);
    free(st.a[l]);
    return OR_OK;
}

/* Kaczmarz pass (Fig. 5) over [e0, e1) of a level vector, against uH. */
int or_kaczmarz(double *v, const double *uH, int e0, int e1) {
    kaczmarz_pass(v, 0, uH, e0, e1);
    return OR_OK;
}

/* One FMG-FAS(-SR) solve, every level stored ("horizontal"): Fig. 2 with the
 * V-cycle of Fig. 1 and the SR changes of Fig. 3 on the SR levels. */
int or_fmg_h(const or_params *p, const double *f, double *u_out) {
    if (check_params(p)) return OR_EINVAL;
    or_state st;
    int rc = alloc_state(&st, p);
    if (rc) return rc;
    rhs_hierarchy(&st, p->M, f);
    rc = fmg_up_to(&st, p->M);
    if (!rc) memcpy(u_out, st.u[p->M], sizeof(double) * ((size_t)1 << p->M));
    free_state(&st);
    return rc;
}

/* `ncycles` FAS V-cycles (Fig. 1) on level M from the iterate u_inout, every
 * level stored; the coarse right-hand sides are rebuilt by each down leg. */
int or_vcycles_h(const or_params *p, const double *f, double *u_inout, int ncycles) {
    if (check_params(p)) return OR_EINVAL;
    or_state st;
    int rc = alloc_state(&st, p);
    if (rc) return rc;
    rhs_hierarchy(&st, p->M, f);
    memcpy(st.u[p->M], u_inout, sizeof(double) * ((size_t)1 << p->M));
    for (int c = 0; c < ncycles && !rc; c++) rc = vcycle(&st, p->M);
    if (!rc) memcpy(u_inout, st.u[p->M], sizeof(double) * ((size_t)1 << p->M));
    free_state(&st);
    return rc;
}

/* The same solve as or_fmg_h, run serially with segmental refinement: the
 * finest level M is never stored.  The FMG steps up to level M-1 run on stored
 * levels.  In the last step each segment of level M is interpolated from level
 * M-1 (Fig. 3 line 1) and smoothed (line 2); its interior is appended to a
 * short window of assembled fine values, from which the restricted solution
 * and the tau-corrected right-hand side of every coarse cell are formed as
 * soon as the six fine cells they read are assembled (lines 3-5), and the
 * window is then trimmed.  After the coarse part of the V-cycle the segment is
 * regenerated from the corrected level M-1 (Eq. 5), smoothed with compatible
 * relaxation and only its interior is emitted (Fig. 3 post-smoothing leg).
 * Memory for level M: one extended patch and a window of at most w + 8 cells.
 * Requires level M to be an SR level, segmented, with tau from the assembled
 * level (tau_src = 0).
 * With post = 1 the post-smoothing leg instead recomputes each segment's
 * pre-smoothed patch from the level M-1 iterate the pre-leg interpolated
 * (kept), puts the neighbouring segments' pre-smoothed interior cells (b + 1 per
 * side, kept from the pre-leg) into its buffer and frozen cells, so that the
 * patch holds the assembled pre-smoothed level, applies the FAS correction of
 * Eq. 4 with the restricted pre-smoothed solution (kept) and smooths without
 * Kaczmarz; then b + 1 <= w is required. */
int or_fmg_v(const or_params *p, const double *f, double *u_out) {
    if (check_params(p)) return OR_EINVAL;
    int M = p->M, n = 1 << M, nc = n / 2;
    if (p->nRS < 1 || !segmented(p, M) || p->tau_src != 0 || M - 1 < p->M0) return OR_EINVAL;
    int w = p->seg_w[M], b = p->seg_b[M];
    if (p->post == 1 && b + 1 > w) return OR_EINVAL;
    const int nseg = n / w, ne = b + 1;   /* post = 1: pre-smoothed cells kept per segment side */
    or_params pc = *p;            /* the stored part: levels M0 .. M-1 */
    pc.M = M - 1;
    pc.nRS = p->nRS - 1;
    or_state st;
    int rc = alloc_state(&st, &pc);
    if (rc) return rc;
    int cap = w + 2 * b + 2, wcap = 2 * w + 16;
    double *patch = (double *)malloc(sizeof(double) * (size_t)cap);
    double *frhs = (double *)malloc(sizeof(double) * (size_t)cap);
    double *win = (double *)malloc(sizeof(double) * (size_t)wcap);
    double *uc_new = (double *)malloc(sizeof(double) * (size_t)nc);
    double *aM = level_coef(p, M);
    double *u_old = NULL, *uhat = NULL, *edge = NULL, *corr = NULL;
    if (p->post == 1) {
        u_old = (double *)malloc(sizeof(double) * (size_t)nc);
        uhat = (double *)malloc(sizeof(double) * (size_t)nc);
        edge = (double *)malloc(sizeof(double) * (size_t)nseg * 2 * ne);
        corr = (double *)malloc(sizeof(double) * (size_t)nc);
    }
    if (!patch || !frhs || !win || !uc_new || (p->op == 2 && !aM) ||
        (p->post == 1 && (!u_old || !uhat || !edge || !corr))) { rc = OR_ENOMEM; goto done; }

    /* right-hand sides of levels M-1 .. M0 (restriction of f), FMG to M-1 */
    for (int J = 0; J < nc; J++) uc_new[J] = restrict_at(f, 0, J);
    rhs_hierarchy(&st, M - 1, uc_new);
    rc = fmg_up_to(&st, M - 1);
    if (rc) goto done;

    /* last step, level M, segment by segment: lines 1-5 of Fig. 3 */
    {
        int win_lo = 0, win_hi = 0;   /* win[i - win_lo] holds assembled cell i */
        int Jnext = 0;                /* next coarse cell whose rhs is pending */
        for (int s = 0; s < n; s += w) {
            int e0, e1, lo, hi;
            extended_patch(s, w, b, n, &e0, &e1, &lo, &hi);
            for (int i = lo; i < hi; i++) {
                patch[i - lo] = prolong_fmg_at(st.u[M - 1], i, nc);
                frhs[i - lo] = f[i];
            }
            patch_sweeps(p->smoother, patch, lo, frhs, lo, n, e0, e1, p->nu1, NULL, op_lam(p), aM);
            if (p->post == 1) {        /* the interior cells the neighbours' patches read */
                memcpy(edge + (size_t)(s / w) * 2 * ne, patch + (s - lo), sizeof(double) * (size_t)ne);
                memcpy(edge + (size_t)(s / w) * 2 * ne + ne, patch + (s + w - ne - lo), sizeof(double) * (size_t)ne);
            }
            memcpy(win + (win_hi - win_lo), patch + (s - lo), sizeof(double) * (size_t)w);
            win_hi += w;
            /* coarse cells whose fine stencil 2J-2 .. 2J+3 is now assembled */
            while (Jnext < nc && (2 * Jnext + 3 < win_hi || win_hi == n)) {
                uc_new[Jnext] = restrict_at(win, win_lo, Jnext);
                st.rhs[M - 1][Jnext] = tau_rhs_at(win, win_lo, f, 0, Jnext, n, op_lam(p), aM, st.a[M - 1]);
                Jnext++;
            }
            /* keep only the cells a pending coarse cell can still read */
            int keep_from = 2 * Jnext - 2 < win_lo ? win_lo : 2 * Jnext - 2;
            memmove(win, win + (keep_from - win_lo), sizeof(double) * (size_t)(win_hi - keep_from));
            win_lo = keep_from;
        }
    }
    if (p->post == 1) {
        memcpy(u_old, st.u[M - 1], sizeof(double) * (size_t)nc);
        memcpy(uhat, uc_new, sizeof(double) * (size_t)nc);
    }
    memcpy(st.u[M - 1], uc_new, sizeof(double) * (size_t)nc);

    /* coarse part of the last V-cycle on the stored levels M-1 .. M0 */
    rc = vcycle(&st, M - 1);
    if (rc) goto done;

    if (p->post == 1) {
        /* post-smoothing leg with the FAS correction (Eq. 4) of the recomputed
         * pre-smoothed segment, S without Kaczmarz, interior emitted */
        for (int J = 0; J < nc; J++) corr[J] = st.u[M - 1][J] - uhat[J];
        for (int s = 0; s < n; s += w) {
            int e0, e1, lo, hi;
            extended_patch(s, w, b, n, &e0, &e1, &lo, &hi);
            for (int i = lo; i < hi; i++) {
                patch[i - lo] = prolong_fmg_at(u_old, i, nc);
                frhs[i - lo] = f[i];
            }
            patch_sweeps(p->smoother, patch, lo, frhs, lo, n, e0, e1, p->nu1, NULL, op_lam(p), aM);
            const int k = s / w;
            if (s > 0)              /* cells [lo, s): the last ne of the left segment */
                for (int i = lo; i < s; i++) patch[i - lo] = edge[(size_t)(k - 1) * 2 * ne + ne + (i - (s - ne))];
            if (s + w < n)          /* cells [s + w, hi): the first ne of the right segment */
                for (int i = s + w; i < hi; i++) patch[i - lo] = edge[(size_t)(k + 1) * 2 * ne + (i - (s + w))];
            for (int i = lo; i < hi; i++) patch[i - lo] += prolong_lin_at(corr, i, nc);
            patch_sweeps(p->smoother, patch, lo, frhs, lo, n, e0, e1, p->nu2, NULL, op_lam(p), aM);
            memcpy(u_out + s, patch + (s - lo), sizeof(double) * (size_t)w);
        }
        goto done;
    }

    /* post-smoothing leg of level M, segment by segment: full update from the
     * corrected level M-1, compatible relaxation, interior emitted */
    for (int s = 0; s < n; s += w) {
        int e0, e1, lo, hi;
        extended_patch(s, w, b, n, &e0, &e1, &lo, &hi);
        for (int i = lo; i < hi; i++) {
            patch[i - lo] = prolong_fmg_at(st.u[M - 1], i, nc);
            frhs[i - lo] = f[i];
        }
        patch_sweeps(p->smoother, patch, lo, frhs, lo, n, e0, e1, p->nu2, st.u[M - 1], op_lam(p), aM);
        memcpy(u_out + s, patch + (s - lo), sizeof(double) * (size_t)w);
    }
done:
    free(patch); free(frhs); free(win); free(uc_new); free(aM);
    free(u_old); free(uhat); free(edge); free(corr);
    free_state(&st);
    return rc;
}
