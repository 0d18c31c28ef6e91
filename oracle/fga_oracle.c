/*
 * fga_oracle.c -- serial FP64 reference ("oracle") for ADMM on a factor graph.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or table with the CUDA
 * path: the factor-type numbers below are an interface both sides agree on
 * and each side writes them down on its own.
 *
 * What it computes (paper: "Testing fine-grained parallelism for the ADMM on
 * a factor-graph", Hao, Oghbaee, Rostami, Derbinsky, Bento):
 *
 *   f(w) = sum_a f_a(w_{da})                               (Sec. II, Eq. 2)
 *   factor graph G=(F,V,E); per edge x,m,u,n, rho, alpha;
 *   per variable z                                          (Sec. II)
 *   one iteration of Algorithm 2, in the paper's order:
 *     for a in F:      x_(a,da) = Prox_{f_a,rho}(n_(a,da))  (x-update)
 *     for (a,b) in E:  m = x + u                            (m-update)
 *     for b in V:      z_b = sum rho m / sum rho            (z-update)
 *     for (a,b) in E:  u = u + alpha (x - z_b)              (u-update)
 *     for (a,b) in E:  n = z_b - u                          (n-update)
 *   Prox_{h,rho}(r) = argmin_s h(s) + rho/2 ||s-r||^2      (Sec. II, Eq. PO)
 *
 * Storage follows the paper's description in Sec. III: edge arrays x,m,u,n
 * in the order the edges were created (factor by factor, each factor's
 * variables in the order given, each variable's components in order); z in
 * the order variables were introduced.  Vector variables are expanded into
 * scalar edges, one per component.
 *
 * Readings where the paper is silent or garbled:
 *   - Sums in the z-update run over a variable's edges in ascending
 *     creation order, sequentially (a canonical order so that a GPU path can
 *     reproduce the sums bit for bit).  Build with -ffp-contract=off.
 *   - Initialisation (unspecified): u = u0 (default 0), n = z0[b] - u.
 *   - Stopping (unspecified, "stopping criteria"): RMS primal residual
 *     sqrt(sum_e (x_e - z_b)^2 / |E|) and RMS dual residual
 *     sqrt(sum_e rho_e^2 (z_b - z_b_prev)^2 / |E|), evaluated after the
 *     n-update of every check_every-th iteration; stop at the first checked
 *     iteration where both are <= their tolerances.
 *   - User-supplied operators (og_register_prox): the paper's addNode
 *     takes each factor's proximal operator as a function pointer
 *     (Sec. III); the x-update calls it with the factor's messages, weights
 *     and parameters in creation order.
 *   - Prox formulas: Appendix A (packing), B (MPC), C (SVM), re-derived
 *     where the printed form has sign or term errors; see each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Factor types (interface numbers, identical on the library side). */
enum {
    OT_PACK_PAIR = 0,        /* no-overlap of two disks, Appendix A          */
    OT_PACK_WALL = 1,        /* disk inside a half-plane, Appendix A          */
    OT_PACK_RADIUS_LIN = 2,  /* f = -w r (linear radius reward)               */
    OT_PACK_RADIUS_QUAD = 3, /* f = -r^2/2 (area reward), Appendix A          */
    OT_SVM_HINGE = 4,        /* f = c max(0, 1 - y (w.x + b))                 */
    OT_SVM_L2 = 5,           /* f = (lambda/2)||w||^2, Appendix C             */
    OT_MPC_DYN = 6,          /* indicator of x' = A x + B u, Appendix B       */
    OT_MPC_QUAD = 7,         /* f = 1/2 sum q_k v_k^2, Appendix B             */
    OT_MPC_BOX = 8,          /* indicator of lo <= v <= hi                    */
    OT_FIX = 9,              /* indicator of v = value                        */
    OT_SVM_MARGIN = 10,      /* indicator of y (w.x + b) >= 1 - xi, App. C    */
    OT_SVM_SLACK = 11,       /* f = lambda sum xi on xi >= 0, Appendix C      */
    OT_EQUAL = 12,           /* indicator of v1 = v2, Appendix C              */
    OT_NTYPES = 13
};

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ESTATE = -4, OR_ENONFINITE = -6 };

/* User-supplied operators.  The paper's addNode receives each factor's
 * proximal operator as a function pointer (Sec. III); og_register_prox does
 * the same here.  fn(arity, n, rho, params, x, ctx) must write
 * x = Prox_{f,rho}(n) (Eq. PO) for one factor: n and rho hold the factor's
 * arity scalar edges in creation order (its variables in the order given,
 * each variable's components in order), params its np parameters.  Types are
 * numbered from OT_USER0 in registration order, per graph. */
typedef void (*og_prox_fn)(int32_t arity, const double *n, const double *rho, const double *params, double *x,
                           void *ctx);
enum { OT_USER0 = 64, OG_MAX_USER = 16 };

typedef struct {
    int32_t type;
    int32_t nv;          /* number of variables                              */
    int64_t var0;        /* offset into g->fvars                              */
    int64_t edge0;       /* first scalar edge (creation order)               */
    int32_t arity;       /* number of scalar edges                            */
    int32_t np;          /* number of parameters                              */
    int64_t par0;        /* offset into g->params                            */
} ofactor;

typedef struct og_graph {
    /* variables */
    int64_t nvar;
    int32_t *vdim;       /* [nvar]                                            */
    int64_t *voff;       /* [nvar] offset of the variable's first component   */
    int64_t nz;          /* scalar variables = sum of dims                    */
    int64_t cap_var;
    /* factors */
    int64_t nfac, cap_fac;
    ofactor *fac;
    int64_t nfvars, cap_fvars;
    int64_t *fvars;      /* variable ids of all factors, concatenated          */
    int64_t nparams, cap_params;
    double *params;
    /* edges (creation order) */
    int64_t ne;
    int64_t *ez;         /* scalar variable of each edge                       */
    double *rho, *alpha;
    double *x, *m, *u, *n;
    double *z, *zprev;
    /* per scalar variable: its edges in ascending creation order */
    int64_t *row;        /* [nz+1]                                             */
    int64_t *col;        /* [ne]                                               */
    int finalized;
    int64_t iters_done;
    double last_rpri, last_rdual;
    /* weight mode: 0 = fixed rho (Algorithm 2 as printed); 1 = three weights
     * (each x-update gives each edge a weight class, see twa_classes) */
    int weights;
    int8_t *cls;         /* [ne] weight class of each edge's last message     */
    /* user-supplied operators, type OT_USER0 + k */
    int32_t nuser;
    og_prox_fn ufn[OG_MAX_USER];
    void *uctx[OG_MAX_USER];
    int32_t uarity[OG_MAX_USER], unp[OG_MAX_USER];
} og_graph;

/* Weight classes of a message (three-weight reading, see og_set_weights). */
enum { OW_ZERO = 0, OW_STD = 1, OW_INF = 2 };

static int grow(void **p, int64_t *cap, int64_t need, size_t elem)
{
    if (need <= *cap) return 0;
    int64_t c = *cap ? *cap : 16;
    while (c < need) c *= 2;
    void *q = realloc(*p, (size_t)c * elem);
    if (!q) return -1;
    *p = q;
    *cap = c;
    return 0;
}

og_graph *og_new(void)
{
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    return g;
}

void og_free(og_graph *g)
{
    if (!g) return;
    free(g->vdim); free(g->voff); free(g->fac); free(g->fvars); free(g->params);
    free(g->ez); free(g->rho); free(g->alpha);
    free(g->x); free(g->m); free(g->u); free(g->n); free(g->z); free(g->zprev);
    free(g->row); free(g->col); free(g->cls);
    free(g);
}

/* Adds `count` variables of dimension `dim`; returns the first id or -1. */
int64_t og_add_vars(og_graph *g, int64_t count, int32_t dim)
{
    if (g->finalized || count < 0 || dim < 1) return -1;
    int64_t cap = g->cap_var;
    if (grow((void **)&g->vdim, &cap, g->nvar + count, sizeof(int32_t))) return -1;
    cap = g->cap_var;
    if (grow((void **)&g->voff, &cap, g->nvar + count, sizeof(int64_t))) return -1;
    g->cap_var = cap;
    int64_t first = g->nvar;
    for (int64_t i = 0; i < count; ++i) {
        g->vdim[g->nvar] = dim;
        g->voff[g->nvar] = g->nz;
        g->nz += dim;
        g->nvar++;
    }
    return first;
}

/* Number of parameters a factor of this type takes, given its variables. */
static int expected_params(int32_t type, int32_t nv, const int32_t *dims, int32_t arity)
{
    switch (type) {
    case OT_PACK_PAIR:
        if (nv != 4 || dims[0] != 2 || dims[1] != 1 || dims[2] != 2 || dims[3] != 1) return -1;
        return 0;
    case OT_PACK_WALL:
        if (nv != 2 || dims[0] != 2 || dims[1] != 1) return -1;
        return 4;
    case OT_PACK_RADIUS_LIN:
        if (nv != 1 || dims[0] != 1) return -1;
        return 1;
    case OT_PACK_RADIUS_QUAD:
        if (nv != 1 || dims[0] != 1) return -1;
        return 0;
    case OT_SVM_HINGE:
        if (nv != 2 || dims[1] != 1) return -1;
        return dims[0] + 2;
    case OT_SVM_L2:
        if (nv != 1) return -1;
        return 1;
    case OT_MPC_DYN:
        if (nv != 3 || dims[0] != dims[2]) return -1;
        return dims[0] * dims[0] + dims[0] * dims[1];
    case OT_MPC_QUAD:
        return arity;
    case OT_MPC_BOX:
        return 2;
    case OT_FIX:
        return arity;
    case OT_SVM_MARGIN:
        if (nv != 3 || dims[1] != 1 || dims[2] != 1) return -1;
        return dims[0] + 1;
    case OT_SVM_SLACK:
        if (nv != 1) return -1;
        return 1;
    case OT_EQUAL:
        if (nv != 2 || dims[0] != dims[1]) return -1;
        return 0;
    default:
        return -1;
    }
}

/* Registers a user-supplied operator for factors of `arity` scalar edges and
 * `np` parameters each; returns its type number (OT_USER0 + k) or -1. */
int32_t og_register_prox(og_graph *g, og_prox_fn fn, void *ctx, int32_t arity, int32_t np)
{
    if (g->finalized || !fn || arity < 1 || np < 0 || g->nuser == OG_MAX_USER) return -1;
    const int32_t k = g->nuser++;
    g->ufn[k] = fn;
    g->uctx[k] = ctx;
    g->uarity[k] = arity;
    g->unp[k] = np;
    return OT_USER0 + k;
}

/* Parameters of a user type for a factor of `arity` scalar edges (-1 if the
 * type is not registered or the arity differs from the registered one). */
static int user_params(const og_graph *g, int32_t type, int32_t arity)
{
    const int32_t k = type - OT_USER0;
    if (k < 0 || k >= g->nuser || g->uarity[k] != arity) return -1;
    return g->unp[k];
}

/* Adds `count` factors of one type.  vars: count*nv variable ids; params:
 * count*np values.  Edges are numbered in call order.  Returns the first
 * factor id or -1. */
int64_t og_add_factors(og_graph *g, int32_t type, int64_t count, int32_t nv,
                       const int64_t *vars, int32_t np, const double *params)
{
    if (g->finalized || count < 0 || nv < 1 || nv > 64) return -1;
    int64_t first = g->nfac;
    for (int64_t f = 0; f < count; ++f) {
        int32_t dims[64];
        int32_t arity = 0;
        for (int32_t k = 0; k < nv; ++k) {
            int64_t v = vars[f * nv + k];
            if (v < 0 || v >= g->nvar) return -1;
            dims[k] = g->vdim[v];
            arity += dims[k];
        }
        const int want = type >= OT_USER0 ? user_params(g, type, arity) : expected_params(type, nv, dims, arity);
        if (want != np) return -1;
        if (grow((void **)&g->fac, &g->cap_fac, g->nfac + 1, sizeof(ofactor))) return -1;
        if (grow((void **)&g->fvars, &g->cap_fvars, g->nfvars + nv, sizeof(int64_t))) return -1;
        if (grow((void **)&g->params, &g->cap_params, g->nparams + np, sizeof(double))) return -1;
        ofactor *a = &g->fac[g->nfac];
        a->type = type;
        a->nv = nv;
        a->var0 = g->nfvars;
        a->edge0 = g->ne;
        a->arity = arity;
        a->np = np;
        a->par0 = g->nparams;
        for (int32_t k = 0; k < nv; ++k) g->fvars[g->nfvars + k] = vars[f * nv + k];
        for (int32_t k = 0; k < np; ++k) g->params[g->nparams + k] = params[f * np + k];
        g->nfvars += nv;
        g->nparams += np;
        g->ne += arity;
        g->nfac++;
    }
    return first;
}

int64_t og_num_edges(const og_graph *g) { return g->ne; }
int64_t og_num_scalar_vars(const og_graph *g) { return g->nz; }

/* Builds the per-edge arrays and each variable's edge list in creation
 * order.  rho = alpha = 1 until og_set_rho_alpha says otherwise. */
int og_finalize(og_graph *g)
{
    if (g->finalized) return OR_ESTATE;
    int64_t E = g->ne, Z = g->nz;
    g->ez = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E ? E : 1));
    g->rho = (double *)malloc(sizeof(double) * (size_t)(E ? E : 1));
    g->alpha = (double *)malloc(sizeof(double) * (size_t)(E ? E : 1));
    g->x = (double *)calloc((size_t)(E ? E : 1), sizeof(double));
    g->m = (double *)calloc((size_t)(E ? E : 1), sizeof(double));
    g->u = (double *)calloc((size_t)(E ? E : 1), sizeof(double));
    g->n = (double *)calloc((size_t)(E ? E : 1), sizeof(double));
    g->z = (double *)calloc((size_t)(Z ? Z : 1), sizeof(double));
    g->zprev = (double *)calloc((size_t)(Z ? Z : 1), sizeof(double));
    g->row = (int64_t *)calloc((size_t)Z + 1, sizeof(int64_t));
    g->col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E ? E : 1));
    g->cls = (int8_t *)malloc((size_t)(E ? E : 1));
    if (!g->ez || !g->rho || !g->alpha || !g->x || !g->m || !g->u || !g->n || !g->z ||
        !g->zprev || !g->row || !g->col || !g->cls)
        return OR_ENOMEM;
    for (int64_t e = 0; e < E; ++e) g->cls[e] = OW_STD;
    for (int64_t a = 0; a < g->nfac; ++a) {
        const ofactor *f = &g->fac[a];
        int64_t e = f->edge0;
        for (int32_t k = 0; k < f->nv; ++k) {
            int64_t v = g->fvars[f->var0 + k];
            for (int32_t c = 0; c < g->vdim[v]; ++c) g->ez[e++] = g->voff[v] + c;
        }
    }
    for (int64_t e = 0; e < E; ++e) {
        g->rho[e] = 1.0;
        g->alpha[e] = 1.0;
        g->row[g->ez[e] + 1]++;
    }
    for (int64_t b = 0; b < Z; ++b) g->row[b + 1] += g->row[b];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(Z ? Z : 1));
    if (!fill) return OR_ENOMEM;
    for (int64_t b = 0; b < Z; ++b) fill[b] = g->row[b];
    for (int64_t e = 0; e < E; ++e) g->col[fill[g->ez[e]]++] = e; /* ascending e */
    free(fill);
    g->finalized = 1;
    return OR_OK;
}

/* rho/alpha: either arrays of |E| values in creation order, or NULL and the
 * uniform values. */
int og_set_rho_alpha(og_graph *g, const double *rho, const double *alpha, double rho_u, double alpha_u)
{
    if (!g->finalized) return OR_ESTATE;
    for (int64_t e = 0; e < g->ne; ++e) {
        double r = rho ? rho[e] : rho_u;
        double a = alpha ? alpha[e] : alpha_u;
        if (!(r > 0.0) || !(a > 0.0)) return OR_EINVAL;
        g->rho[e] = r;
        g->alpha[e] = a;
    }
    return OR_OK;
}

/* Weight mode.  The paper keeps rho and alpha fixed per edge and notes that
 * improved update schemes exist which its framework can run (Sec. II, the
 * three-weight algorithm of Derbinsky et al.); it states none.  Reading
 * (mode 1, "three weights"): each x-update gives each of the factor's edges
 * a weight class --
 *   infinite: the factor fixes the value whatever it receives (FIX);
 *   zero: a constraint-type factor (disk pair, wall, box, hinge, margin)
 *         whose proximal step left that edge's message unchanged (the
 *         constraint does not act on it: no opinion);
 *   standard: every other edge;
 * the z-update averages only the infinite-weight messages m if there are
 * any, else the standard ones with weights rho, else (all zero) all of them
 * as in mode 0; and the u-update sets u = 0 on an edge of zero or infinite
 * weight (a fixed value's scaled dual, and an inactive constraint's, are
 * zero) and runs u += alpha (x - z) on the others. */
int og_set_weights(og_graph *g, int32_t mode)
{
    if (!g->finalized) return OR_ESTATE;
    if (mode != 0 && mode != 1) return OR_EINVAL;
    g->weights = mode;
    for (int64_t e = 0; e < g->ne; ++e) g->cls[e] = OW_STD;
    return OR_OK;
}

/* Initialisation (reading of the unspecified start): z = z0 (default 0),
 * u = u0 (default 0), n = z_b - u, x = m = 0. */
int og_init(og_graph *g, const double *z0, const double *u0)
{
    if (!g->finalized) return OR_ESTATE;
    for (int64_t b = 0; b < g->nz; ++b) g->z[b] = z0 ? z0[b] : 0.0;
    for (int64_t e = 0; e < g->ne; ++e) {
        g->u[e] = u0 ? u0[e] : 0.0;
        g->x[e] = 0.0;
        g->m[e] = 0.0;
        g->n[e] = g->z[g->ez[e]] - g->u[e];
    }
    g->iters_done = 0;
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Proximal operators (Eq. PO), one per factor type.  n: the factor's
 * incoming messages (arity values, creation order), rho: the matching edge
 * weights, p: parameters, dims: variable dimensions.  Writes x.
 * ------------------------------------------------------------------------ */

/* Appendix A, no-collision: minimise sum_k rho_k/2 |v_k - n_k|^2 subject to
 * ||c1 - c2|| >= r1 + r2, variables (c1 in R^2, r1, c2 in R^2, r2).
 * The constraint only involves c1-c2 along their current direction and
 * r1+r2, so the solution moves c1 by -t1 nhat, c2 by +t2 nhat and both radii
 * down by t_r, with sum t = D = max(0, r1 + r2 - |c1 - c2|) split in
 * proportion to 1/rho.  The printed form has "+1" on the radius component;
 * growing the radii would deepen the overlap, so the radius moves by -t
 * (reading checked against a brute-force minimiser in the tests).  Equal
 * rho gives the printed magnitude D/2 * rho2/(rho1+rho2).  When the centres
 * coincide the direction is taken as nhat = (1, 0). */
static void prox_pack_pair(const double *n, const double *rho, double *x)
{
    double dx = n[3] - n[0];
    double dy = n[4] - n[1];
    double d = sqrt(dx * dx + dy * dy);
    double D = n[2] + n[5] - d;
    if (!(D > 0.0)) {
        for (int k = 0; k < 6; ++k) x[k] = n[k];
        return;
    }
    double hx = 1.0, hy = 0.0;
    if (d > 0.0) {
        hx = dx / d;
        hy = dy / d;
    }
    double wc1 = 1.0 / rho[0], wr1 = 1.0 / rho[2];
    double wc2 = 1.0 / rho[3], wr2 = 1.0 / rho[5];
    double W = wc1 + wr1 + wc2 + wr2;
    double tc1 = (D * wc1) / W, tr1 = (D * wr1) / W;
    double tc2 = (D * wc2) / W, tr2 = (D * wr2) / W;
    x[0] = n[0] - tc1 * hx;
    x[1] = n[1] - tc1 * hy;
    x[2] = n[2] - tr1;
    x[3] = n[3] + tc2 * hx;
    x[4] = n[4] + tc2 * hy;
    x[5] = n[5] - tr2;
}

/* Appendix A, wall: minimise rho_c/2 |c - n_c|^2 + rho_r/2 (r - n_r)^2
 * subject to Q.(c - V) >= r.  Params (Qx, Qy, Vx, Vy).  If the constraint
 * holds at n, x = n; otherwise the Lagrange condition gives
 * c = n_c + lam w_c Q, r = n_r - lam w_r with
 * lam = -h / (w_c |Q|^2 + w_r), h = Q.(n_c - V) - n_r, w = 1/rho.  With
 * |Q| = 1 and equal rho this is the printed (c,r) = n + E(-Q, 1),
 * E = min(0, h/2). */
static void prox_pack_wall(const double *n, const double *rho, const double *p, double *x)
{
    double Qx = p[0], Qy = p[1], Vx = p[2], Vy = p[3];
    double h = Qx * (n[0] - Vx) + Qy * (n[1] - Vy) - n[2];
    if (h >= 0.0) {
        x[0] = n[0];
        x[1] = n[1];
        x[2] = n[2];
        return;
    }
    double wc = 1.0 / rho[0], wr = 1.0 / rho[2];
    double den = wc * (Qx * Qx + Qy * Qy) + wr;
    double lam = -h / den;
    double sc = lam * wc;
    x[0] = n[0] + sc * Qx;
    x[1] = n[1] + sc * Qy;
    x[2] = n[2] - lam * wr;
}

/* Linear radius reward f = -w r: argmin -w r + rho/2 (r - n)^2 = n + w/rho. */
static void prox_pack_radius_lin(const double *n, const double *rho, const double *p, double *x)
{
    x[0] = n[0] + p[0] / rho[0];
}

/* Appendix A, area reward f = -r^2/2: argmin = rho n / (rho - 1); the
 * minimisation is bounded only for rho > 1 (checked at iterate time). */
static void prox_pack_radius_quad(const double *n, const double *rho, double *x)
{
    x[0] = (rho[0] * n[0]) / (rho[0] - 1.0);
}

/* Hinge f = c max(0, 1 - y (w.x + b)) on (w in R^D, b); params (x[D], y, c).
 * This is the slack-free form of Appendix C's one-point margin operator:
 * with t = 1 - y (n_w.x + n_b) and s = sum_j x_j^2/rho_wj + 1/rho_b, the
 * step along (y x, y) weighted by 1/rho is gamma = min(c, t/s) when t > 0,
 * else 0. */
static void prox_svm_hinge(int32_t D, const double *n, const double *rho, const double *p, double *x)
{
    const double *xi = p;
    double y = p[D], c = p[D + 1];
    double dot = 0.0, s = 0.0;
    for (int32_t j = 0; j < D; ++j) dot += n[j] * xi[j];
    dot += n[D];
    for (int32_t j = 0; j < D; ++j) s += (xi[j] * xi[j]) / rho[j];
    s += 1.0 / rho[D];
    double t = 1.0 - y * dot;
    if (!(t > 0.0)) {
        for (int32_t j = 0; j <= D; ++j) x[j] = n[j];
        return;
    }
    double gam = t / s;
    if (gam > c) gam = c;
    double gy = gam * y;
    for (int32_t j = 0; j < D; ++j) x[j] = n[j] + (gy * xi[j]) / rho[j];
    x[D] = n[D] + gy / rho[D];
}

/* Appendix C, minimal norm two, with weight lambda:
 * argmin lambda/2 |w|^2 + rho/2 |w - n|^2 = rho n / (rho + lambda). */
static void prox_svm_l2(int32_t arity, const double *n, const double *rho, const double *p, double *x)
{
    for (int32_t j = 0; j < arity; ++j) x[j] = (rho[j] * n[j]) / (rho[j] + p[0]);
}

/* Appendix C, one-point minimal margin: the indicator of
 * y (w.x + b) >= 1 - xi on v = (w in R^d, b, xi); params x[d], y.  Its prox
 * is the rho-weighted projection onto the half-space a.v >= 1 with
 * a = (y x, y, 1):
 *     v = n + lambda W a,   lambda = (1 - a.n)^+ / (a^T W a),   W = diag(1/rho).
 * (The printed closed form inverts the sign of the violation, writes
 * n1.w + n2 b for n1.x + n2, drops y from the b update and moves w, b, xi
 * against a; this is the projection the stated problem defines.) */
static void prox_svm_margin(int32_t d, const double *n, const double *rho, const double *p, double *x)
{
    const double y = p[d];
    double an = 0.0, awa = 0.0;
    for (int32_t j = 0; j < d; ++j) {
        const double aj = y * p[j];
        an += aj * n[j];
        awa += (aj * aj) / rho[j];
    }
    an += y * n[d];
    awa += (y * y) / rho[d];
    an += n[d + 1];
    awa += 1.0 / rho[d + 1];
    const double viol = 1.0 - an;
    const double lam = viol > 0.0 ? viol / awa : 0.0;
    for (int32_t j = 0; j < d; ++j) x[j] = n[j] + (lam * (y * p[j])) / rho[j];
    x[d] = n[d] + (lam * y) / rho[d];
    x[d + 1] = n[d + 1] + lam / rho[d + 1];
}

/* Appendix C, minimal error: argmin lambda xi + rho/2 (xi - n)^2 over
 * xi >= 0, per component: xi = (n - lambda/rho)^+. */
static void prox_svm_slack(int32_t arity, const double *n, const double *rho, const double *p, double *x)
{
    for (int32_t j = 0; j < arity; ++j) {
        const double v = n[j] - p[0] / rho[j];
        x[j] = v > 0.0 ? v : 0.0;
    }
}

/* Appendix C, equality of two copies v1, v2 in R^d: both become the
 * rho-weighted mean, per component. */
static void prox_equal(int32_t d, const double *n, const double *rho, double *x)
{
    for (int32_t j = 0; j < d; ++j) {
        const double v = (rho[j] * n[j] + rho[d + j] * n[d + j]) / (rho[j] + rho[d + j]);
        x[j] = v;
        x[d + j] = v;
    }
}

/* Dense Cholesky solve of an SPD k x k system (in place), used by the
 * dynamics projection below. */
static int chol_solve(int k, double *K, double *b)
{
    for (int j = 0; j < k; ++j) {
        double s = K[j * k + j];
        for (int i = 0; i < j; ++i) s -= K[j * k + i] * K[j * k + i];
        if (!(s > 0.0)) return -1;
        double l = sqrt(s);
        K[j * k + j] = l;
        for (int r = j + 1; r < k; ++r) {
            double t = K[r * k + j];
            for (int i = 0; i < j; ++i) t -= K[r * k + i] * K[j * k + i];
            K[r * k + j] = t / l;
        }
    }
    for (int r = 0; r < k; ++r) { /* L y = b */
        double t = b[r];
        for (int i = 0; i < r; ++i) t -= K[r * k + i] * b[i];
        b[r] = t / K[r * k + r];
    }
    for (int r = k - 1; r >= 0; --r) { /* L^T x = y */
        double t = b[r];
        for (int i = r + 1; i < k; ++i) t -= K[i * k + r] * b[i];
        b[r] = t / K[r * k + r];
    }
    return 0;
}

/* Appendix B, linearised dynamics: the indicator of x_{t+1} = A x_t + B u_t
 * on v = (x_t, u_t, x_{t+1}), i.e. of M v = 0 with M = [A  B  -I].  Its
 * prox is the rho-weighted projection
 *     v = n - W M^T (M W M^T)^{-1} M n,   W = diag(1/rho).
 * (The printed objective omits the constraint; this is the reading.) */
static int prox_mpc_dyn(int32_t nx, int32_t nu, const double *n, const double *rho, const double *p, double *x)
{
    const double *A = p, *B = p + nx * nx;
    int32_t nvv = 2 * nx + nu;
    double *M = (double *)malloc(sizeof(double) * (size_t)(nx * nvv));
    double *K = (double *)malloc(sizeof(double) * (size_t)(nx * nx));
    double *r = (double *)malloc(sizeof(double) * (size_t)nx);
    if (!M || !K || !r) { free(M); free(K); free(r); return OR_ENOMEM; }
    for (int32_t i = 0; i < nx; ++i) {
        for (int32_t j = 0; j < nx; ++j) M[i * nvv + j] = A[i * nx + j];
        for (int32_t j = 0; j < nu; ++j) M[i * nvv + nx + j] = B[i * nu + j];
        for (int32_t j = 0; j < nx; ++j) M[i * nvv + nx + nu + j] = (i == j) ? -1.0 : 0.0;
    }
    for (int32_t i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < nvv; ++j) s += M[i * nvv + j] * n[j];
        r[i] = s;
        for (int32_t k = 0; k < nx; ++k) {
            double t = 0.0;
            for (int32_t j = 0; j < nvv; ++j) t += M[i * nvv + j] * M[k * nvv + j] / rho[j];
            K[i * nx + k] = t;
        }
    }
    int rc = chol_solve(nx, K, r);
    if (rc == 0) {
        for (int32_t j = 0; j < nvv; ++j) {
            double t = 0.0;
            for (int32_t i = 0; i < nx; ++i) t += M[i * nvv + j] * r[i];
            x[j] = n[j] - t / rho[j];
        }
    }
    free(M); free(K); free(r);
    return rc == 0 ? OR_OK : OR_EINVAL;
}

/* Appendix B, diagonal quadratic cost f = 1/2 sum q_k v_k^2:
 * v_k = rho_k n_k / (q_k + rho_k), the rho (Q + rho I)^{-1} n form. */
static void prox_mpc_quad(int32_t arity, const double *n, const double *rho, const double *p, double *x)
{
    for (int32_t j = 0; j < arity; ++j) x[j] = (rho[j] * n[j]) / (p[j] + rho[j]);
}

/* Box indicator lo <= v <= hi: projection = clamp. */
static void prox_mpc_box(int32_t arity, const double *n, const double *p, double *x)
{
    double lo = p[0], hi = p[1];
    for (int32_t j = 0; j < arity; ++j) {
        double v = n[j];
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        x[j] = v;
    }
}

/* Equality indicator v = value: the prox returns the value. */
static void prox_fix(int32_t arity, const double *p, double *x)
{
    for (int32_t j = 0; j < arity; ++j) x[j] = p[j];
}

/* Public single-factor prox, for tests.  dims: the nv variable dimensions. */
int og_prox(int32_t type, int32_t nv, const int32_t *dims, const double *params,
            const double *rho, const double *n, double *x)
{
    int32_t arity = 0;
    for (int32_t k = 0; k < nv; ++k) arity += dims[k];
    switch (type) {
    case OT_PACK_PAIR: prox_pack_pair(n, rho, x); return OR_OK;
    case OT_PACK_WALL: prox_pack_wall(n, rho, params, x); return OR_OK;
    case OT_PACK_RADIUS_LIN: prox_pack_radius_lin(n, rho, params, x); return OR_OK;
    case OT_PACK_RADIUS_QUAD:
        if (!(rho[0] > 1.0)) return OR_EINVAL;
        prox_pack_radius_quad(n, rho, x);
        return OR_OK;
    case OT_SVM_HINGE: prox_svm_hinge(dims[0], n, rho, params, x); return OR_OK;
    case OT_SVM_L2: prox_svm_l2(arity, n, rho, params, x); return OR_OK;
    case OT_MPC_DYN: return prox_mpc_dyn(dims[0], dims[1], n, rho, params, x);
    case OT_MPC_QUAD: prox_mpc_quad(arity, n, rho, params, x); return OR_OK;
    case OT_MPC_BOX: prox_mpc_box(arity, n, params, x); return OR_OK;
    case OT_FIX: prox_fix(arity, params, x); return OR_OK;
    case OT_SVM_MARGIN: prox_svm_margin(dims[0], n, rho, params, x); return OR_OK;
    case OT_SVM_SLACK: prox_svm_slack(arity, n, rho, params, x); return OR_OK;
    case OT_EQUAL: prox_equal(dims[0], n, rho, x); return OR_OK;
    default: return OR_EINVAL;
    }
}

static int factor_prox(og_graph *g, const ofactor *f)
{
    if (f->type >= OT_USER0) {
        /* the user's operator, through its function pointer */
        const int32_t k = f->type - OT_USER0;
        g->ufn[k](f->arity, g->n + f->edge0, g->rho + f->edge0, g->params + f->par0, g->x + f->edge0, g->uctx[k]);
        return OR_OK;
    }
    int32_t dims[64];
    for (int32_t k = 0; k < f->nv; ++k) dims[k] = g->vdim[g->fvars[f->var0 + k]];
    return og_prox(f->type, f->nv, dims, g->params + f->par0, g->rho + f->edge0,
                   g->n + f->edge0, g->x + f->edge0);
}

/* Runs Algorithm 2 until max_iters iterations have been done in this call
 * or the residuals of a checked iteration are both within tolerance.
 * Returns the number of iterations done and the last residuals (RMS). */
/* Weight classes of factor f's edges after its x-update (mode 1). */
static void twa_classes(og_graph *g, const ofactor *f)
{
    for (int32_t k = 0; k < f->arity; ++k) {
        const int64_t e = f->edge0 + k;
        int8_t c = OW_STD;
        if (f->type == OT_FIX) {
            c = OW_INF;
        } else if (f->type == OT_PACK_PAIR || f->type == OT_PACK_WALL || f->type == OT_MPC_BOX ||
                   f->type == OT_SVM_HINGE || f->type == OT_SVM_MARGIN) {
            if (g->x[e] == g->n[e]) c = OW_ZERO;
        }
        g->cls[e] = c;
    }
}

int og_iterate(og_graph *g, int64_t max_iters, double tol_pri, double tol_dual,
               int32_t check_every, int64_t *iters_out, double *rpri_out, double *rdual_out)
{
    if (!g->finalized) return OR_ESTATE;
    if (check_every < 1) check_every = 1;
    int64_t E = g->ne, Z = g->nz;
    double rpri = NAN, rdual = NAN;
    int64_t it = 0;
    int status = OR_OK;
    while (it < max_iters) {
        /* x-update: one proximal operator per factor */
        for (int64_t a = 0; a < g->nfac; ++a) {
            int rc = factor_prox(g, &g->fac[a]);
            if (rc != OR_OK) return rc;
            if (g->weights) twa_classes(g, &g->fac[a]);
        }
        /* m-update */
        for (int64_t e = 0; e < E; ++e) g->m[e] = g->x[e] + g->u[e];
        /* z-update: rho-weighted average over each variable's edges */
        if (!g->weights) {
            for (int64_t b = 0; b < Z; ++b) {
                double S = 0.0, R = 0.0;
                for (int64_t k = g->row[b]; k < g->row[b + 1]; ++k) {
                    int64_t e = g->col[k];
                    S += g->rho[e] * g->m[e];
                    R += g->rho[e];
                }
                g->zprev[b] = g->z[b];
                if (R > 0.0) g->z[b] = S / R; /* a variable with no edge keeps z */
            }
        } else {
            /* three weights: infinite-weight messages first, then standard
             * ones, then all of them (each sum in ascending edge order) */
            for (int64_t b = 0; b < Z; ++b) {
                double S = 0.0, R = 0.0, Ss = 0.0, Rs = 0.0, Si = 0.0, Ni = 0.0;
                for (int64_t k = g->row[b]; k < g->row[b + 1]; ++k) {
                    int64_t e = g->col[k];
                    if (g->cls[e] == OW_INF) {
                        Si += g->m[e];
                        Ni += 1.0;
                    } else {
                        S += g->rho[e] * g->m[e];
                        R += g->rho[e];
                        if (g->cls[e] == OW_STD) {
                            Ss += g->rho[e] * g->m[e];
                            Rs += g->rho[e];
                        }
                    }
                }
                g->zprev[b] = g->z[b];
                if (Ni > 0.0) g->z[b] = Si / Ni;
                else if (Rs > 0.0) g->z[b] = Ss / Rs;
                else if (R > 0.0) g->z[b] = S / R;
            }
        }
        /* u-update */
        if (!g->weights) {
            for (int64_t e = 0; e < E; ++e) g->u[e] = g->u[e] + g->alpha[e] * (g->x[e] - g->z[g->ez[e]]);
        } else {
            for (int64_t e = 0; e < E; ++e)
                g->u[e] = g->cls[e] == OW_STD ? g->u[e] + g->alpha[e] * (g->x[e] - g->z[g->ez[e]]) : 0.0;
        }
        /* n-update */
        for (int64_t e = 0; e < E; ++e) g->n[e] = g->z[g->ez[e]] - g->u[e];
        ++it;
        g->iters_done++;
        if (g->iters_done % check_every == 0 || it == max_iters) {
            double sp = 0.0, sd = 0.0;
            for (int64_t e = 0; e < E; ++e) {
                int64_t b = g->ez[e];
                double r = g->x[e] - g->z[b];
                double s = g->rho[e] * (g->z[b] - g->zprev[b]);
                sp += r * r;
                sd += s * s;
            }
            rpri = E ? sqrt(sp / (double)E) : 0.0;
            rdual = E ? sqrt(sd / (double)E) : 0.0;
            if (!isfinite(rpri) || !isfinite(rdual)) {
                status = OR_ENONFINITE;
                break;
            }
            if (rpri <= tol_pri && rdual <= tol_dual) break;
        }
    }
    g->last_rpri = rpri;
    g->last_rdual = rdual;
    if (iters_out) *iters_out = it;
    if (rpri_out) *rpri_out = rpri;
    if (rdual_out) *rdual_out = rdual;
    return status;
}

/* Readout: which = 0 x, 1 m, 2 u, 3 n (creation order); z in variable order. */
int og_get_edge(const og_graph *g, int32_t which, double *out)
{
    if (!g->finalized) return OR_ESTATE;
    const double *src = which == 0 ? g->x : which == 1 ? g->m : which == 2 ? g->u : which == 3 ? g->n : NULL;
    if (!src) return OR_EINVAL;
    memcpy(out, src, sizeof(double) * (size_t)g->ne);
    return OR_OK;
}

int og_get_z(const og_graph *g, double *out)
{
    if (!g->finalized) return OR_ESTATE;
    memcpy(out, g->z, sizeof(double) * (size_t)g->nz);
    return OR_OK;
}

/* Scalar variable of each edge (creation order). */
int og_get_edge_var(const og_graph *g, int64_t *out)
{
    if (!g->finalized) return OR_ESTATE;
    memcpy(out, g->ez, sizeof(int64_t) * (size_t)g->ne);
    return OR_OK;
}
