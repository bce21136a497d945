/*
 * pmp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the
 * particle-mesh-particle (PMP) cycle of He, Wibking, Vijayan, Krumholz & Li,
 * "A novel algorithm for GPU-accelerated particle-mesh interactions
 * implemented in the Quokka code" (arXiv:2509.18261):
 *
 *   Sec. 2.1      problem statement, kernel of radius r_K about the particle
 *   Sec. 2.2      Steps 1-5 (buffer deposit, ghost sum, limiter, particle
 *                 update, mesh update)
 *   Sec. 3.1.1    sink accretion (Eqs. rbh, mdot, kernel, kernel_wgt,
 *                 truelove, accretion_function, and the accretion limiter)
 *   Sec. 3.2.1    supernova feedback (Eq. du, v_COM, Eq. dp, Eq. psnr, and
 *                 the momentum limiter Eq. lambda)
 *   App. A.2      ghost contributions summed in a fixed order
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file.  The library under paper_2509_18261_gb300/ never links it and
 * shares no code with it.  Loops run over particles in index order, then over
 * stencil cells in lexicographic order (z slowest, x fastest), then over mesh
 * cells.
 *
 * Build without fused multiply-add (gcc -ffp-contract=off): every product and
 * sum written below is rounded on its own, in the order written, except where
 * the code calls fma() (C99; x * y + z rounded once).
 *
 * Reading (evaluation): the paper fixes FP64 but no evaluation order.  A
 * product that is added to a running sum or to another term is fused with
 * that addition where the code says fma(): the gather sums of Sec. 3.2.1 and
 * the sum of kernel weights of Eq. kernel_wgt, the momentum and energy rows of
 * Eq. du, and the Step-4 sums of Sec. 2.2.  Every quotient by rho in the sink
 * formulas of Sec. 3.1.1 (the Delta U rows, v in Step 4, c_s^2) is a product
 * with the cell's one reciprocal 1/rho; the auxiliary fields and sink
 * creation keep their divisions.  Everything else is rounded operation by
 * operation.
 *
 * Readings of points the paper leaves open are marked "Reading:".
 * Parity unpinned: the sub-sampled covered fraction omega and the code-unit
 * constants A_sf, A_p have no values printed in the paper; the tests check
 * them only by self-consistency (symmetry, convergence, conservation, the
 * 0.46 E_sn calibration).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NF 5
#define OR_PI 3.141592653589793

enum { KIND_FEEDBACK = 0, KIND_SINK = 1, KIND_MASS = 2 };

/* status codes returned by every entry point */
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OUTSIDE = 2, OR_ERR_NONFINITE = 3, OR_ERR_NOMEM = 4 };

typedef struct {
    int32_t kind;      /* 0 supernova feedback, 1 sink accretion */
    int32_t subsample; /* S: sub-points per axis for the covered fraction omega */
    double r_K;        /* kernel radius, cell units (Sec. 2.1) */
    double dt;         /* time step (Eq. accretion_function) */
    double G;          /* gravitational constant (Eq. rbh, Eq. truelove) */
    double gamma;      /* adiabatic index of the ideal gas */
    double lambda_bh;  /* lambda of Eq. mdot */
    double J;          /* Jeans number of Eq. truelove */
    double cap;        /* largest fraction of a cell's mass removed per step */
    double rho_min;    /* density floor */
    double A_sf;       /* M_sf = A_sf n_H^-0.26 (code units) */
    double A_p;        /* P_snr = A_p n_H^-0.17 (code units) */
    double mu_H;       /* mass per H nucleus */
    double RM_ej;      /* R_M <= RM_ej: EJ regime */
    double RM_st;      /* RM_ej < R_M <= RM_st: ST regime; above: MC */
    double eps_K;      /* kinetic fraction in the ST regime (Eq. dp) */
} or_params;

typedef struct {
    int32_t n[3];        /* valid cells per axis */
    int32_t ng;          /* ghost cells on every side */
    int32_t periodic[3]; /* 1: axis wraps; 0: kernels are cut at the faces;
                            2: the ghost cells hold the values of the cells
                            they stand for (a patch of a batch, whose ghosts
                            were filled from its neighbours) */
    int32_t pad_;
    double dx;           /* physical cell size; V = dx^3 */
    int64_t fstride;     /* doubles between fields */
    double *u;           /* [5][fstride], padded box, x fastest */
} or_mesh;

typedef struct {
    int64_t count;
    const double *x, *y, *z; /* cell units, 0 <= x < n */
    double *m;               /* feedback: ejecta mass; sink: sink mass */
    double *px, *py, *pz;    /* momentum (feedback: ejecta momentum) */
    const double *e;         /* feedback: supernova energy; sink: unused */
} or_particles;

/* ------------------------------------------------------------------------ */
/* Elementary functions.  exp and log are written out here (instead of the C  */
/* library's) so that the CUDA path, which implements the same published      */
/* methods independently, can reproduce every bit.                            */
/* ------------------------------------------------------------------------ */

/* ln 2 split for Cody & Waite (1980) argument reduction: LN2_HI keeps the top
 * 32 significant bits of ln 2 (so k*LN2_HI is exact for |k| < 2^21) and
 * LN2_LO is the next 53 bits of ln 2 = 0.693147180559945309417232121458...
 * The published fdlibm library prints the same split (and the log
 * arrangement f - (hf - s (hf + R)) used below); the polynomials are this
 * oracle's own. */
static const double LN2_HI = 6.93147180369123816490e-01;
static const double LN2_LO = 1.90821492927058770002e-10;
static const double INV_LN2 = 1.44269504088896338700e+00;

/* 2^k for any integer k, as an exact power of two where representable. */
static double pow2i(int k)
{
    double r = 1.0;
    while (k > 0) { int s = k > 60 ? 60 : k; r = r * (double)(1ULL << s); k -= s; }
    while (k < 0) { int s = -k > 60 ? 60 : -k; r = r / (double)(1ULL << s); k += s; }
    return r;
}

/* exp(x): Cody & Waite reduction x = k ln2 + r, |r| <= ln2/2, then the Taylor
 * series of e^r to degree 13 (truncation error < 4e-18 relative) by Horner's
 * rule, then scaling by 2^k. */
double or_exp(double x)
{
    if (x != x) return x;
    if (x > 709.79) return INFINITY;
    if (x < -745.2) return 0.0;
    double kd = floor(x * INV_LN2 + 0.5);
    int k = (int)kd;
    double r = (x - kd * LN2_HI) - kd * LN2_LO;
    /* coefficients 1/j! (j! is exact in double for j <= 13) */
    double fact = 1.0;
    double c[14];
    c[0] = 1.0;
    for (int j = 1; j <= 13; j++) { fact = fact * (double)j; c[j] = 1.0 / fact; }
    double p = c[13];
    for (int j = 12; j >= 0; j--) p = p * r + c[j];
    if (k < -1000) return (p * pow2i(k + 200)) * pow2i(-200);
    if (k > 1000) return (p * pow2i(k - 200)) * pow2i(200);
    return p * pow2i(k);
}

/* log(x), x > 0: x = 2^e (1 + f) with 1 + f in [sqrt(1/2), sqrt(2)), then
 * log(1 + f) = 2 atanh(s), s = f / (2 + f), |s| <= 0.1716.  Writing
 * 2 atanh(s) = 2s + s R(z), z = s^2, R(z) = sum_{j=1..11} 2 z^j / (2j + 1)
 * (truncation < 1e-18 relative), and using the identity 2s = f - s f =
 * f - hf + s hf with hf = f^2 / 2:
 *   log(1 + f) = f - (hf - s (hf + R)),
 * whose leading term f is exact.  log x = e ln2 + log(1 + f), small terms
 * first. */
double or_log(double x)
{
    if (x != x || x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (isinf(x)) return x;
    int e;
    double m = frexp(x, &e); /* x = m 2^e, m in [0.5, 1) */
    m = m * 2.0;
    e = e - 1;
    if (m > 1.4142135623730951) { m = m * 0.5; e = e + 1; }
    double f = m - 1.0;
    double s = f / (2.0 + f);
    double z = s * s;
    double R = 2.0 / 23.0;
    for (int j = 10; j >= 1; j--) R = R * z + 2.0 / (double)(2 * j + 1);
    R = R * z;
    double hf = 0.5 * (f * f);
    double ed = (double)e;
    return ed * LN2_HI - ((hf - (s * (hf + R) + ed * LN2_LO)) - f);
}

/* x^a for x > 0 through the two functions above. */
double or_pow(double x, double a) { return or_exp(a * or_log(x)); }

/* ------------------------------------------------------------------------ */
/* Mesh helpers                                                              */
/* ------------------------------------------------------------------------ */

static int64_t cell_index(const or_mesh *M, int i, int j, int k)
{
    int64_t px = (int64_t)M->n[0] + 2 * M->ng;
    int64_t py = (int64_t)M->n[1] + 2 * M->ng;
    return ((int64_t)(k + M->ng) * py + (int64_t)(j + M->ng)) * px + (int64_t)(i + M->ng);
}

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* conserved state (rho, px, py, pz, E) of a valid cell */
static void read_state(const or_mesh *S, int i, int j, int k, double U[NF])
{
    int64_t c = cell_index(S, i, j, k);
    for (int f = 0; f < NF; f++) U[f] = S->u[(int64_t)f * S->fstride + c];
}

/* Sec. 2.1: the kernel is measured from cell centres; in cell units the
 * centre of cell i is at i + 1/2. */
static double centre_offset(int c, double x) { return ((double)c + 0.5) - x; }

/* Reading (Sec. 2.1 writes "> r_K" for zero, Sec. 3.2.1 "< r_K" for inside):
 * a cell belongs to the kernel iff |x_c - x_s|^2 < r_K^2, the squared
 * distance summed as (dx^2 + dy^2) + dz^2. */
static int inside(double d2, double r2) { return d2 < r2; }

static int stencil_halfwidth(double rK) { return (int)ceil(rK); }

/* Reading of "the fraction of the grid cell that is covered by the stencil"
 * (Sec. 3.2.1): the share of the S^3 mid-points of an S x S x S sub-grid of
 * the cell that lie strictly inside r_K, counted only for cells whose centre
 * lies inside (the same cells V_snr sums over).  S = 1 gives omega = 1. */
static int64_t covered_subpoints(int S, double r2, int ci, int cj, int ck, double x, double y, double z)
{
    int64_t cnt = 0;
    for (int c = 0; c < S; c++)
        for (int b = 0; b < S; b++)
            for (int a = 0; a < S; a++) {
                double sx = ((double)ci + ((double)a + 0.5) / (double)S) - x;
                double sy = ((double)cj + ((double)b + 0.5) / (double)S) - y;
                double sz = ((double)ck + ((double)c + 0.5) / (double)S) - z;
                double d2 = (sx * sx + sy * sy) + sz * sz;
                if (inside(d2, r2)) cnt++;
            }
    return cnt;
}

/* One kernel cell as enumerated for a particle: unwrapped index, the wrapped
 * (owning) valid index, centre offsets, squared distance. */
typedef struct {
    int ci, cj, ck;       /* unwrapped buffer coordinates */
    int wi, wj, wk;       /* owning valid cell */
    double d[3];
    double d2;
} kcell;

/* Enumerates kernel cells of a particle in canonical order (z slowest).  On a
 * non-periodic axis the kernel is cut at the domain face (cells outside the
 * domain are not part of it).  Returns the count written to out. */
static int kernel_cells(const or_mesh *S, double rK, double x, double y, double z, kcell *out)
{
    int R = stencil_halfwidth(rK);
    double r2 = rK * rK;
    int hx = (int)floor(x), hy = (int)floor(y), hz = (int)floor(z);
    int cnt = 0;
    for (int oz = -R; oz <= R; oz++)
        for (int oy = -R; oy <= R; oy++)
            for (int ox = -R; ox <= R; ox++) {
                int ci = hx + ox, cj = hy + oy, ck = hz + oz;
                if (!S->periodic[0] && (ci < 0 || ci >= S->n[0])) continue;
                if (!S->periodic[1] && (cj < 0 || cj >= S->n[1])) continue;
                if (!S->periodic[2] && (ck < 0 || ck >= S->n[2])) continue;
                double d0 = centre_offset(ci, x), d1 = centre_offset(cj, y), d2c = centre_offset(ck, z);
                double dd = (d0 * d0 + d1 * d1) + d2c * d2c;
                if (!inside(dd, r2)) continue;
                kcell *kc = &out[cnt++];
                kc->ci = ci; kc->cj = cj; kc->ck = ck;
                kc->wi = S->periodic[0] == 2 ? ci : wrap(ci, S->n[0]);
                kc->wj = S->periodic[1] == 2 ? cj : wrap(cj, S->n[1]);
                kc->wk = S->periodic[2] == 2 ? ck : wrap(ck, S->n[2]);
                kc->d[0] = d0; kc->d[1] = d1; kc->d[2] = d2c;
                kc->d2 = dd;
            }
    return cnt;
}

static int check_position(const or_mesh *S, double x, double y, double z)
{
    if (!(x == x && y == y && z == z)) return OR_ERR_NONFINITE;
    if (!(x >= 0.0 && x < (double)S->n[0])) return OR_ERR_OUTSIDE;
    if (!(y >= 0.0 && y < (double)S->n[1])) return OR_ERR_OUTSIDE;
    if (!(z >= 0.0 && z < (double)S->n[2])) return OR_ERR_OUTSIDE;
    return OR_OK;
}

static double cell_volume(double dx) { return (dx * dx) * dx; }

/* ------------------------------------------------------------------------ */
/* Sink per-cell quantities (Sec. 3.1.1)                                     */
/* ------------------------------------------------------------------------ */

/* Ideal-gas sound speed squared c_s^2 = gamma (gamma - 1) e_int / rho with
 * e_int = E - |p|^2 / (2 rho) (clamped at 0), and the Truelove density
 * rho_Tr = J^2 pi c_s^2 / (G dx^2) (Eq. truelove).  Reading (evaluation):
 * every quotient by rho in the sink formulas of Sec. 3.1.1 is a product with
 * the cell's one reciprocal inv = 1/rho, so e_int = E - |p|^2 (inv/2) and
 * c_s^2 = (gamma (gamma - 1) e_int) inv. */
static void sink_cell(const or_params *P, double dx, const double U[NF], double *cs, double *rho_tr)
{
    double inv = 1.0 / U[0];
    double ke2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3];
    double eint = U[4] - ke2 * (0.5 * inv);
    if (eint < 0.0) eint = 0.0;
    double gg = P->gamma * (P->gamma - 1.0);
    double cs2 = (gg * eint) * inv;
    double ctr = ((P->J * P->J) * OR_PI) / (P->G * (dx * dx));
    *cs = sqrt(cs2);
    *rho_tr = ctr * cs2;
}

/* Gathered rows, [rows][count] */
#define FB_ROWS 12
#define SK_ROWS 8
#define MS_ROWS 6
#define MAX_ROWS 12
enum { FB_MSNR = 0, FB_VSNR, FB_VX, FB_VY, FB_VZ, FB_NH, FB_RM, FB_PRAD, FB_Q, FB_E, FB_PV, FB_REGIME };
enum { SK_RHO = 0, SK_VINF, SK_CINF, SK_MDOT, SK_RACC, SK_SUMW, SK_K, SK_NMEM };
enum { MS_VK = 0, MS_Q };  /* V_K, then the five per-volume amounts q_f */

int or_gathered_rows(int kind) { return kind == KIND_FEEDBACK ? FB_ROWS : (kind == KIND_SINK ? SK_ROWS : MS_ROWS); }

static kcell *alloc_kcells(double rK)
{
    int R = stencil_halfwidth(rK);
    int64_t w = 2 * (int64_t)R + 1;
    return (kcell *)malloc(sizeof(kcell) * (size_t)(w * w * w));
}

/* ------------------------------------------------------------------------ */
/* Gather (particle side of Step 1): feedback                               */
/* ------------------------------------------------------------------------ */

/* Sec. 3.2.1: M_snr = sum omega rho V + M_ej, V_snr = sum omega V, v_COM,
 * n_H = M_snr / (mu_H V_snr), R_M = M_snr / M_sf with M_sf = A_sf n_H^-0.26,
 * the regime and |p_radial| of Eq. dp / Eq. psnr.
 * Readings: V_snr carries omega like M_snr; M_ej v_ej is the particle's
 * momentum; E_kin = |p|^2 / (2 M_ej); V is the same for every cell of a box,
 * so sums run over omega rho and omega p and are multiplied by V once. */
static int gather_feedback_one(const or_params *P, const or_mesh *S, const or_particles *p, int64_t s,
                               kcell *kc, double *G, int64_t stride)
{
    double x = p->x[s], y = p->y[s], z = p->z[s];
    int st = check_position(S, x, y, z);
    if (st) return st;
    double m = p->m[s], pe[3] = {p->px[s], p->py[s], p->pz[s]}, Esn = p->e[s];
    if (!(m > 0.0)) return OR_ERR_NONFINITE;
    int S3 = P->subsample * P->subsample * P->subsample;
    double r2 = P->r_K * P->r_K;
    int nk = kernel_cells(S, P->r_K, x, y, z, kc);
    double sw = 0.0, sr = 0.0, sp[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < nk; t++) {
        int64_t cnt = covered_subpoints(P->subsample, r2, kc[t].ci, kc[t].cj, kc[t].ck, x, y, z);
        if (cnt == 0) continue;
        double w = (double)cnt / (double)S3;
        double U[NF];
        read_state(S, kc[t].wi, kc[t].wj, kc[t].wk, U);
        sw = sw + w;
        sr = fma(w, U[0], sr);
        for (int a = 0; a < 3; a++) sp[a] = fma(w, U[1 + a], sp[a]);
    }
    double V = cell_volume(S->dx);
    double Vsnr = sw * V;
    double Mgas = sr * V;
    double Msnr = Mgas + m;
    double vc[3];
    for (int a = 0; a < 3; a++) vc[a] = (sp[a] * V + pe[a]) / Msnr;
    double nH = Msnr / (P->mu_H * Vsnr);
    double Msf = P->A_sf * or_pow(nH, -0.26);
    double RM = Msnr / Msf;
    int regime;
    double prad;
    if (RM <= P->RM_ej) { regime = 0; prad = 0.0; }                                   /* EJ */
    else if (RM <= P->RM_st) { regime = 1; prad = sqrt(((2.0 * m) * P->eps_K) * Esn); } /* ST */
    else { regime = 2; prad = P->A_p * or_pow(nH, -0.17); }                           /* MC */
    double vej2 = (pe[0] * pe[0] + pe[1] * pe[1]) + pe[2] * pe[2];
    double Ekin = vej2 / (2.0 * m);
    G[FB_MSNR * stride] = Msnr;
    G[FB_VSNR * stride] = Vsnr;
    G[FB_VX * stride] = vc[0];
    G[FB_VY * stride] = vc[1];
    G[FB_VZ * stride] = vc[2];
    G[FB_NH * stride] = nH;
    G[FB_RM * stride] = RM;
    G[FB_PRAD * stride] = prad;
    G[FB_Q * stride] = m / Vsnr;
    G[FB_E * stride] = (Esn + Ekin) / Vsnr;
    G[FB_PV * stride] = prad / Vsnr;
    G[FB_REGIME * stride] = (double)regime;
    if (!isfinite(Msnr) || !isfinite(nH) || !isfinite(prad) || !isfinite(Ekin)) return OR_ERR_NONFINITE;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Gather: sink                                                              */
/* ------------------------------------------------------------------------ */

/* Gaussian weight factor of one axis, Eq. kernel written as a product over
 * axes: exp(-r^2/r_acc^2) = prod_a exp(-d_a^2 / r_acc^2). */
static double axis_weight(double d, double ra2) { return or_exp(-((d * d) / ra2)); }

static double kernel_weight(const kcell *c, double ra2)
{
    return (axis_weight(c->d[0], ra2) * axis_weight(c->d[1], ra2)) * axis_weight(c->d[2], ra2);
}

/* Sec. 3.1.1: rho_inf (mean density over the kernel), v_inf = |sum m_c (v_c
 * - v_s)| / sum m_c and c_inf = sum m_c c_s,c / sum m_c (mass-weighted), then
 * r_BH (Eq. rbh), mdot_BH (Eq. mdot), r_acc and sum w (Eq. kernel).
 * Readings: m_c v_c is the cell momentum p_c V; V is common to all cells and
 * cancels from the weighted means; r_acc is in cell units (r_BH / dx). */
static int gather_sink_one(const or_params *P, const or_mesh *S, const or_particles *p, int64_t s,
                           kcell *kc, double *G, int64_t stride)
{
    double x = p->x[s], y = p->y[s], z = p->z[s];
    int st = check_position(S, x, y, z);
    if (st) return st;
    double ms = p->m[s], ps[3] = {p->px[s], p->py[s], p->pz[s]};
    if (!(ms > 0.0)) return OR_ERR_NONFINITE;
    int nk = kernel_cells(S, P->r_K, x, y, z, kc);
    double srho = 0.0, sp[3] = {0.0, 0.0, 0.0}, src = 0.0;
    for (int t = 0; t < nk; t++) {
        double U[NF], cs, rtr;
        read_state(S, kc[t].wi, kc[t].wj, kc[t].wk, U);
        sink_cell(P, S->dx, U, &cs, &rtr);
        srho = srho + U[0];
        for (int a = 0; a < 3; a++) sp[a] = sp[a] + U[1 + a];
        src = src + U[0] * cs;
    }
    double rho_inf = srho / (double)nk;
    double c_inf = src / srho;
    double u[3];
    for (int a = 0; a < 3; a++) u[a] = sp[a] / srho - ps[a] / ms;
    double vinf2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    double cinf2 = c_inf * c_inf;
    double den = vinf2 + cinf2;
    double r_bh = (P->G * ms) / den;
    double lam2 = P->lambda_bh * P->lambda_bh;
    double mdot = (((4.0 * OR_PI) * rho_inf) * (r_bh * r_bh)) * sqrt(lam2 * cinf2 + vinf2);
    double racc = r_bh / S->dx;
    if (racc < 0.25) racc = 0.25;
    if (racc > 0.5 * P->r_K) racc = 0.5 * P->r_K;
    double ra2 = racc * racc;
    double sumw = 0.0;
    for (int t = 0; t < nk; t++)
        sumw = fma(axis_weight(kc[t].d[0], ra2) * axis_weight(kc[t].d[1], ra2), axis_weight(kc[t].d[2], ra2), sumw);
    double V = cell_volume(S->dx);
    double K = ((mdot * P->dt) / V) / sumw;
    G[SK_RHO * stride] = rho_inf;
    G[SK_VINF * stride] = sqrt(vinf2);
    G[SK_CINF * stride] = c_inf;
    G[SK_MDOT * stride] = mdot;
    G[SK_RACC * stride] = racc;
    G[SK_SUMW * stride] = sumw;
    G[SK_K * stride] = K;
    G[SK_NMEM * stride] = (double)nk;
    if (!(den > 0.0) || !isfinite(mdot) || !isfinite(K)) { G[SK_K * stride] = 0.0; return OR_ERR_NONFINITE; }
    return OR_OK;
}

/* Particle-mesh (PM/PIC) deposit, the step subset of Sec. 2.2 that uses Steps
 * 1, 2 and 5 only: a particle spreads its mass, momentum and energy content
 * over its kernel cells in proportion to the covered fraction omega.
 * Reading: the paper names no assignment function for this use; the kernel
 * and omega are those of the supernova deposit (Sec. 3.2.1), so that
 * sum_c Delta U_c V returns (m, p, e) and no cell outside r_K is touched.
 * V_K = sum omega V; q_f = (m, p_x, p_y, p_z, e)_f / V_K (e = 0 if the
 * particles carry no energy). */
static int gather_mass_one(const or_params *P, const or_mesh *S, const or_particles *p, int64_t s, kcell *kc,
                           double *G, int64_t stride)
{
    double x = p->x[s], y = p->y[s], z = p->z[s];
    int st = check_position(S, x, y, z);
    if (st) return st;
    int S3 = P->subsample * P->subsample * P->subsample;
    double r2 = P->r_K * P->r_K;
    int nk = kernel_cells(S, P->r_K, x, y, z, kc);
    double sw = 0.0;
    for (int t = 0; t < nk; t++) {
        int64_t cnt = covered_subpoints(P->subsample, r2, kc[t].ci, kc[t].cj, kc[t].ck, x, y, z);
        if (cnt == 0) continue;
        sw = sw + (double)cnt / (double)S3;
    }
    double VK = sw * cell_volume(S->dx);
    double u[NF] = {p->m[s], p->px[s], p->py[s], p->pz[s], p->e ? p->e[s] : 0.0};
    G[MS_VK * stride] = VK;
    for (int f = 0; f < NF; f++) G[(MS_Q + f) * stride] = u[f] / VK;
    return OR_OK;
}

static int gather_one(const or_params *P, const or_mesh *S, const or_particles *p, int64_t s, kcell *kc, double *G,
                      int64_t stride)
{
    if (P->kind == KIND_FEEDBACK) return gather_feedback_one(P, S, p, s, kc, G, stride);
    if (P->kind == KIND_SINK) return gather_sink_one(P, S, p, s, kc, G, stride);
    return gather_mass_one(P, S, p, s, kc, G, stride);
}

int or_gather(const or_params *P, const or_mesh *S, const or_particles *p, double *gathered)
{
    if (!P || !S || !p || !gathered) return OR_ERR_ARG;
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return OR_ERR_NOMEM;
    int status = OR_OK;
    for (int64_t s = 0; s < p->count; s++) {
        int st = gather_one(P, S, p, s, kc, gathered + s, p->count);
        if (st && !status) status = st;
    }
    free(kc);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Deposition functions Delta U^s_c                                          */
/* ------------------------------------------------------------------------ */

/* Eq. du with the readings:
 *   drho = omega q,                                   q = M_ej / V_snr
 *   dp   = omega ((rho_c + q) v_COM - p_c) + p_rad,c
 *   dE   = omega e + v_COM . p_rad,c,                 e = (E_sn + E_kin) / V_snr
 *   p_rad,c = (omega |p_radial| / V_snr) d / |d|,     d = x_c - x_s (0 if d = 0)
 * Momentum smoothing acts on the covered part (fraction omega) of the cell,
 * whose density after the ejecta arrive is rho_c + q; with omega in {0, 1}
 * this is the printed row.  Sums over the kernel then give exactly M_ej,
 * M_ej v_ej + sum p_rad,c V, and E_sn + E_kin + v_COM . sum p_rad,c V. */
static void feedback_delta(double w, const double U[NF], const double *G, int64_t stride, const kcell *c,
                           double dU[NF])
{
    double q = G[FB_Q * stride], e = G[FB_E * stride], Pv = G[FB_PV * stride];
    double vc[3] = {G[FB_VX * stride], G[FB_VY * stride], G[FB_VZ * stride]};
    double rn = U[0] + q;
    double dist = sqrt(c->d2);
    double s = c->d2 > 0.0 ? (w * Pv) / dist : 0.0;
    double pr[3];
    for (int a = 0; a < 3; a++) pr[a] = s * c->d[a];
    dU[0] = w * q;
    for (int a = 0; a < 3; a++) dU[1 + a] = fma(w, fma(rn, vc[a], -U[1 + a]), pr[a]);
    dU[4] = fma(w, e, fma(vc[2], pr[2], fma(vc[1], pr[1], vc[0] * pr[0])));
}

/* Eq. accretion_function with the Truelove rate folded into the max:
 * removal a = max(mdot_BH phi dt / V, rho - rho_Tr), written as
 * max(K w, rho - rho_Tr) with K = mdot_BH dt / V / sum w, and
 * Delta U = -a (1, v, e_sp + v^2/2) = -a (1, p/rho, E/rho), each quotient a
 * product with inv = 1/rho (reading above). */
static void sink_delta(const or_params *P, double dx, const double U[NF], const double *G, int64_t stride,
                       const kcell *c, double dU[NF])
{
    double racc = G[SK_RACC * stride], K = G[SK_K * stride];
    double w = kernel_weight(c, racc * racc);
    double cs, rtr;
    sink_cell(P, dx, U, &cs, &rtr);
    double bh = K * w;
    double tr = U[0] - rtr;
    double a = bh >= tr ? bh : tr;
    double inv = 1.0 / U[0];
    dU[0] = -a;
    for (int k = 0; k < 3; k++) dU[1 + k] = -(a * (U[1 + k] * inv));
    dU[4] = -(a * (U[4] * inv));
}

/* Particle-mesh deposit: Delta U_c = omega q (every row). */
static void mass_delta(double w, const double *G, int64_t stride, double dU[NF])
{
    for (int f = 0; f < NF; f++) dU[f] = w * G[(MS_Q + f) * stride];
}

/* Delta U^s_c of the context's kind (w = omega; 1 for sinks). */
static void kind_delta(const or_params *P, double dx, double w, const double U[NF], const double *G, int64_t stride,
                       const kcell *c, double dU[NF])
{
    if (P->kind == KIND_FEEDBACK) feedback_delta(w, U, G, stride, c, dU);
    else if (P->kind == KIND_SINK) sink_delta(P, dx, U, G, stride, c, dU);
    else mass_delta(w, G, stride, dU);
}

/* Covered fraction of a kernel cell (1 for sinks). */
static double cell_fraction(const or_params *P, const kcell *c, double x, double y, double z)
{
    if (P->kind == KIND_SINK) return 1.0;
    int S = P->subsample;
    int64_t cnt = covered_subpoints(S, P->r_K * P->r_K, c->ci, c->cj, c->ck, x, y, z);
    return (double)cnt / (double)(S * S * S);
}

/* ------------------------------------------------------------------------ */
/* Step 1: deposit into the buffer (Eq. delta_u_buf)                         */
/* ------------------------------------------------------------------------ */

/* buf += sum_s Delta U^s, particles in index order, kernel cells in canonical
 * order, each added at its unwrapped buffer index (ghosts included).  When
 * absbuf is given, it accumulates sum_s |Delta U^s| per cell and field (the
 * analogue of the error buffer E of App. A.1, used for tolerances).  Cells
 * with omega = 0 receive nothing. */
static int deposit_parts(const or_params *P, const or_mesh *S, const or_particles *p, const double *gathered,
                         int64_t gstride, or_mesh *B, double *absbuf);
static int deposit_parts_e(const or_params *P, const or_mesh *S, const or_particles *p, const double *gathered,
                           int64_t gstride, or_mesh *B, double *absbuf, double *ebuf);

int or_deposit(const or_params *P, const or_mesh *S, const or_particles *p, const double *gathered, or_mesh *B,
               double *absbuf)
{
    if (!P || !S || !p || !gathered || !B) return OR_ERR_ARG;
    if (B->ng < stencil_halfwidth(P->r_K)) return OR_ERR_ARG;
    return deposit_parts(P, S, p, gathered, p->count, B, absbuf);
}

/* App. A.1, step 4: a buffer value v with error bound e keeps all but its
 * least significant N_bit = log2(e / |v|) + 52 + M significand bits.
 * Reading: log2 is rounded up to an integer (ceil, taken exactly from the
 * binary exponent), N_bit is clamped to [0, 52], the dropped bits are set to
 * zero (truncation toward zero), and v = 0 or e = 0 is left as it is. */
static double repro_round(double v, double e, int M)
{
    if (v == 0.0 || !(e > 0.0)) return v;
    double r = e / fabs(v);
    if (!(r > 0.0)) return v;
    int nbit;
    if (r >= 1.0) {
        nbit = 52;
    } else {
        int k;
        double m = frexp(r, &k); /* r = m 2^k, 1/2 <= m < 1, so k - 1 <= log2 r < k */
        int ceil_log2 = (m == 0.5) ? k - 1 : k;
        nbit = ceil_log2 + 52 + M;
        if (nbit < 0) nbit = 0;
        if (nbit > 52) nbit = 52;
    }
    uint64_t bits;
    memcpy(&bits, &v, sizeof bits);
    if (nbit > 0) bits &= ~((((uint64_t)1) << nbit) - 1);
    memcpy(&v, &bits, sizeof v);
    return v;
}

/* App. A.1 (reproducible atomics), steps 1-4: Step 1 as or_deposit, with an
 * error bound per buffer value, E := E + eps |Delta U^buf| after every
 * addition (eps = 2^-52, the FP64 machine epsilon); then every buffer value
 * (ghost cells included) rounded by repro_round with margin M.  ebuf (same
 * layout as the buffer, zeroed by the caller) returns E. */
int or_deposit_rounded(const or_params *P, const or_mesh *S, const or_particles *p, const double *gathered,
                       or_mesh *B, int M, double *ebuf)
{
    if (!P || !S || !p || !gathered || !B || !ebuf || M < 0) return OR_ERR_ARG;
    if (B->ng < stencil_halfwidth(P->r_K)) return OR_ERR_ARG;
    int st = deposit_parts_e(P, S, p, gathered, p->count, B, NULL, ebuf);
    int64_t ncell = (int64_t)(B->n[0] + 2 * B->ng) * (B->n[1] + 2 * B->ng) * (B->n[2] + 2 * B->ng);
    for (int f = 0; f < NF; f++)
        for (int64_t c = 0; c < ncell; c++) {
            int64_t o = (int64_t)f * B->fstride + c;
            B->u[o] = repro_round(B->u[o], ebuf[o], M);
        }
    return st;
}

/* or_deposit with particle s's gathered row r at gathered[r * gstride + s]. */
static int deposit_parts(const or_params *P, const or_mesh *S, const or_particles *p, const double *gathered,
                         int64_t gstride, or_mesh *B, double *absbuf)
{
    return deposit_parts_e(P, S, p, gathered, gstride, B, absbuf, NULL);
}

static int deposit_parts_e(const or_params *P, const or_mesh *S, const or_particles *p, const double *gathered,
                           int64_t gstride, or_mesh *B, double *absbuf, double *ebuf)
{
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return OR_ERR_NOMEM;
    int status = OR_OK;
    for (int64_t s = 0; s < p->count; s++) {
        double x = p->x[s], y = p->y[s], z = p->z[s];
        int st = check_position(S, x, y, z);
        if (st) { if (!status) status = st; continue; }
        int nk = kernel_cells(S, P->r_K, x, y, z, kc);
        for (int t = 0; t < nk; t++) {
            double w = cell_fraction(P, &kc[t], x, y, z);
            if (w == 0.0) continue;
            double U[NF], dU[NF];
            read_state(S, kc[t].wi, kc[t].wj, kc[t].wk, U);
            kind_delta(P, S->dx, w, U, gathered + s, gstride, &kc[t], dU);
            int64_t b = cell_index(B, kc[t].ci, kc[t].cj, kc[t].ck);
            for (int f = 0; f < NF; f++) {
                int64_t o = (int64_t)f * B->fstride + b;
                B->u[o] = B->u[o] + dU[f];
                if (absbuf) absbuf[o] = absbuf[o] + fabs(dU[f]);
                if (ebuf) ebuf[o] = ebuf[o] + 2.220446049250313e-16 * fabs(B->u[o]);
            }
        }
    }
    free(kc);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Step 2: ghost-zone summation on one box                                   */
/* ------------------------------------------------------------------------ */

/* Each valid cell c becomes ((B_c + B_img1) + B_img2) + ... over its ghost
 * images c + o n (o in {-1,0,1}^3 without 0, periodic axes only, image inside
 * the padded box), images taken in lexicographic order of (oz, oy, ox): a
 * fixed summation order for cells with several contributors (App. A.2).
 * Requires ng <= n on every axis. */
static void fold_field(const or_mesh *B, double *u)
{
    int nx = B->n[0], ny = B->n[1], nz = B->n[2], g = B->ng;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int64_t c = cell_index(B, i, j, k);
                double v = u[c];
                for (int oz = -1; oz <= 1; oz++)
                    for (int oy = -1; oy <= 1; oy++)
                        for (int ox = -1; ox <= 1; ox++) {
                            if (ox == 0 && oy == 0 && oz == 0) continue;
                            if ((ox && !B->periodic[0]) || (oy && !B->periodic[1]) || (oz && !B->periodic[2])) continue;
                            int gi = i + ox * nx, gj = j + oy * ny, gk = k + oz * nz;
                            if (gi < -g || gi >= nx + g || gj < -g || gj >= ny + g || gk < -g || gk >= nz + g) continue;
                            v = v + u[cell_index(B, gi, gj, gk)];
                        }
                u[c] = v;
            }
}

int or_fold(or_mesh *B, double *absbuf)
{
    if (!B) return OR_ERR_ARG;
    for (int a = 0; a < 3; a++)
        if (B->ng > B->n[a]) return OR_ERR_ARG;
    for (int f = 0; f < NF; f++) {
        fold_field(B, B->u + (int64_t)f * B->fstride);
        if (absbuf) fold_field(B, absbuf + (int64_t)f * B->fstride);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 3: limiters                                                          */
/* ------------------------------------------------------------------------ */

/* Supernova momentum limiter (Eq. lambda).  Reading: T is the pre-deposit
 * temperature, so C_V (rho + drho) T = e_int0 (rho + drho) / rho with
 * e_int0 = E - |p|^2 / (2 rho).  lambda = 1 if the constraint holds at 1;
 * else the largest root in [0, 1] of
 *   |dp|^2 l^2 + 2 (p . dp) l + |p|^2 - 2 rho' (E' - e_int0 rho' / rho) = 0,
 * from the cancellation-free quadratic formula of Press et al., Numerical
 * Recipes, Sec. 5.6; lambda = 0 when no root lies in [0, 1].  Only momentum
 * is scaled: eta = (1, l, l, l, 1).  *noroot is set when lambda = 0 had to be
 * taken. */
static double sn_lambda(const double U[NF], const double D[NF], int *noroot)
{
    *noroot = 0;
    if (D[1] == 0.0 && D[2] == 0.0 && D[3] == 0.0) return 1.0;
    double rho1 = U[0] + D[0];
    double E1 = U[4] + D[4];
    double p2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3];
    double eint0 = U[4] - p2 / (2.0 * U[0]);
    double pn[3];
    for (int a = 0; a < 3; a++) pn[a] = U[1 + a] + D[1 + a];
    double pn2 = (pn[0] * pn[0] + pn[1] * pn[1]) + pn[2] * pn[2];
    double therm = (eint0 * rho1) / U[0];
    double lhs = therm + pn2 / (2.0 * rho1);
    if (lhs <= E1) return 1.0;
    double A = (D[1] * D[1] + D[2] * D[2]) + D[3] * D[3];
    if (!(A > 0.0)) return 1.0;
    double B = (U[1] * D[1] + U[2] * D[2]) + U[3] * D[3];
    double C = p2 - (2.0 * rho1) * (E1 - therm);
    double disc = B * B - A * C;
    if (!(disc >= 0.0)) { *noroot = 1; return 0.0; }
    double sq = sqrt(disc);
    double hi, lo;
    if (B >= 0.0) {
        double Q = -(B + sq);
        hi = Q != 0.0 ? C / Q : 0.0;
        lo = Q / A;
    } else {
        double Q = sq - B;
        hi = Q / A;
        lo = C / Q;
    }
    if (hi < 0.0 || lo > 1.0) { *noroot = 1; return 0.0; }
    return hi < 1.0 ? hi : 1.0;
}

/* Accretion limiter (Sec. 3.1.1) composed with the density floor: with the
 * removal a = -drho,
 *   a_lim = min(max(min(a, cap rho), rho - rho_Tr), rho - rho_min), >= 0,
 * eta = a_lim / a if a_lim < a, else 1; the same eta for all fields.  With
 * cap = 1/4 and rho_min = 0 this is the printed limiter. */
static double sink_eta(const or_params *P, double dx, const double U[NF], const double D[NF])
{
    double a = -D[0];
    if (!(a > 0.0)) return 1.0;
    double cs, rtr;
    sink_cell(P, dx, U, &cs, &rtr);
    double rho = U[0];
    double al = a < P->cap * rho ? a : P->cap * rho;
    double t = rho - rtr;
    al = al > t ? al : t;
    double f = rho - P->rho_min;
    al = al < f ? al : f;
    if (al < 0.0) al = 0.0;
    return al < a ? al / a : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Step 4: limited changes returned to sink particles                        */
/* ------------------------------------------------------------------------ */

/* One cell's terms of the Step-4 sums: with a = -Delta U_rho (the removal of
 * Eq. accretion_function) and b = eta a, the mass sum takes -b and the
 * momentum sums take -b v with v = p inv, inv = 1/rho, fused (Reading
 * (evaluation)). */
static void return_add(double eta, const double U[NF], const double dU[NF], double acc[4])
{
    double b = eta * (-dU[0]);
    double inv = 1.0 / U[0];
    acc[0] = acc[0] - b;
    for (int k = 0; k < 3; k++) acc[1 + k] = fma(-b, U[1 + k] * inv, acc[1 + k]);
}

/* u_s := u_s - sum_c eta_c Delta U^s_c V, with Delta U^s recomputed exactly as
 * in Step 1 and eta from the pre-update state and the summed buffer of the
 * owning cell (eta at a ghost image is its owner's).  V is common to all
 * cells, so u_s := u_s - V sum_c eta_c Delta U^s_c. */
static int return_parts(const or_params *P, const or_mesh *S, const or_mesh *B, or_particles *p,
                        const double *gathered, int64_t gstride);

int or_return_sinks(const or_params *P, const or_mesh *S, const or_mesh *B, or_particles *p, const double *gathered)
{
    if (!P || !S || !B || !p || !gathered || P->kind != KIND_SINK) return OR_ERR_ARG;
    return return_parts(P, S, B, p, gathered, p->count);
}

/* or_return_sinks with particle s's gathered row r at gathered[r * gstride + s]. */
static int return_parts(const or_params *P, const or_mesh *S, const or_mesh *B, or_particles *p,
                        const double *gathered, int64_t gstride)
{
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return OR_ERR_NOMEM;
    double V = cell_volume(S->dx);
    int status = OR_OK;
    for (int64_t s = 0; s < p->count; s++) {
        double x = p->x[s], y = p->y[s], z = p->z[s];
        int st = check_position(S, x, y, z);
        if (st) { if (!status) status = st; continue; }
        int nk = kernel_cells(S, P->r_K, x, y, z, kc);
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = 0; t < nk; t++) {
            double U[NF], dU[NF], D[NF];
            read_state(S, kc[t].wi, kc[t].wj, kc[t].wk, U);
            sink_delta(P, S->dx, U, gathered + s, gstride, &kc[t], dU);
            int64_t o = cell_index(B, kc[t].wi, kc[t].wj, kc[t].wk);
            for (int f = 0; f < NF; f++) D[f] = B->u[(int64_t)f * B->fstride + o];
            double eta = sink_eta(P, S->dx, U, D);
            return_add(eta, U, dU, acc);
        }
        p->m[s] = p->m[s] - acc[0] * V;
        p->px[s] = p->px[s] - acc[1] * V;
        p->py[s] = p->py[s] - acc[2] * V;
        p->pz[s] = p->pz[s] - acc[3] * V;
    }
    free(kc);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Steps 3 + 5: limiter and mesh update                                      */
/* ------------------------------------------------------------------------ */

/* U := U + eta Delta U^sum on every valid cell.  eta_out (optional, one value
 * per valid cell, x fastest) receives the momentum eta for feedback and the
 * common eta for sinks.  counts[0] = cells with eta < 1, counts[1] = cells
 * where no admissible lambda existed (feedback).
 * Reading: a cell whose summed change is zero in every field receives
 * nothing and is left as it is (eta = 1 there); the floating-point sum
 * U + 0 would differ from U only by turning a -0 into +0. */
static int all_zero(const double D[NF])
{
    for (int f = 0; f < NF; f++)
        if (D[f] != 0.0) return 0;
    return 1;
}

/* Step 3 of the context's kind: eta per field of one cell (Eq. lambda for
 * supernovae, the accretion limiter for sinks, 1 for the particle-mesh
 * deposit, which Sec. 2.2 leaves unlimited). */
static void kind_eta(const or_params *P, double dx, const double U[NF], const double D[NF], double eta[NF], int *nr)
{
    *nr = 0;
    if (P->kind == KIND_FEEDBACK) {
        double l = sn_lambda(U, D, nr);
        eta[0] = 1.0; eta[1] = l; eta[2] = l; eta[3] = l; eta[4] = 1.0;
    } else if (P->kind == KIND_SINK) {
        double e = sink_eta(P, dx, U, D);
        for (int f = 0; f < NF; f++) eta[f] = e;
    } else {
        for (int f = 0; f < NF; f++) eta[f] = 1.0;
    }
}

int or_apply(const or_params *P, or_mesh *S, const or_mesh *B, double *eta_out, int64_t *counts)
{
    if (!P || !S || !B) return OR_ERR_ARG;
    int64_t n_lim = 0, n_noroot = 0, v = 0;
    for (int k = 0; k < S->n[2]; k++)
        for (int j = 0; j < S->n[1]; j++)
            for (int i = 0; i < S->n[0]; i++, v++) {
                double U[NF], D[NF];
                int64_t c = cell_index(S, i, j, k), b = cell_index(B, i, j, k);
                for (int f = 0; f < NF; f++) {
                    U[f] = S->u[(int64_t)f * S->fstride + c];
                    D[f] = B->u[(int64_t)f * B->fstride + b];
                }
                double eta[NF];
                int nr;
                kind_eta(P, S->dx, U, D, eta, &nr);
                n_noroot += nr;
                if (eta[1] < 1.0) n_lim++;
                if (eta_out) eta_out[v] = eta[1];
                if (all_zero(D)) continue;
                for (int f = 0; f < NF; f++) S->u[(int64_t)f * S->fstride + c] = U[f] + eta[f] * D[f];
            }
    if (counts) { counts[0] = n_lim; counts[1] = n_noroot; }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Auxiliary conserved fields under accretion (Sec. 3.1.1, extensions)       */
/* ------------------------------------------------------------------------ */

/* The dual-energy internal energy density and species densities follow the
 * accretion function with e_sp + v^2/2 replaced by their value per unit mass
 * (Delta rho_sp = (rho_sp / rho) Delta rho): each pair's change is -a X/rho
 * with the cell's X/rho.  Reading: that common factor is taken out of the sum
 * over particles, Delta X^sum = (X/rho) Delta rho^sum, and the limiter's eta
 * applies as to every other field: X := X + eta ((X / rho) Delta rho^sum), on
 * the pre-update state (before Step 5).  X: [n][stride] with the state's cell
 * layout. */
int or_apply_extra(const or_params *P, const or_mesh *S, const or_mesh *B, double *X, int n, int64_t stride)
{
    if (!P || !S || !B || (n > 0 && !X) || P->kind != KIND_SINK) return OR_ERR_ARG;
    for (int k = 0; k < S->n[2]; k++)
        for (int j = 0; j < S->n[1]; j++)
            for (int i = 0; i < S->n[0]; i++) {
                double U[NF], D[NF];
                read_state(S, i, j, k, U);
                int64_t b = cell_index(B, i, j, k), c = cell_index(S, i, j, k);
                for (int f = 0; f < NF; f++) D[f] = B->u[(int64_t)f * B->fstride + b];
                if (all_zero(D)) continue;
                double eta = sink_eta(P, S->dx, U, D);
                for (int f = 0; f < n; f++) {
                    double x = X[(int64_t)f * stride + c];
                    X[(int64_t)f * stride + c] = x + eta * ((x / U[0]) * D[0]);
                }
            }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sink creation (Sec. 3.1.2)                                                */
/* ------------------------------------------------------------------------ */

/* After the accretion pass, with its summed buffer B retained (Sec. 3.1, item
 * 2), a valid cell c becomes a new sink when
 *   (a) rho_c > rho_Tr,c (Eq. truelove with the cell's own c_s);
 *   (b) c is a local density maximum within r_K: rho_c > rho_c' for every
 *       other valid cell c' whose centre lies within r_K of c's centre;
 *   (c) no sink lies within r_K, enforced as the paper does: the summed
 *       change of the accretion pass is zero in every field at c.
 * Readings: "within r_K" is |x_c' - x_c|^2 < r_K^2 with the cell-centre
 * offsets of Sec. 2.1, periodic images on periodic axes; the maximum is
 * strict (equal neighbours create nothing); all conditions are evaluated on
 * the state before any creation.  Then, in cell index order (z slowest), the
 * sink gets position = the cell centre, m_s = (rho - rho_Tr) V and p_s =
 * m_s v with v = p_c / rho_c; the cell keeps its velocity and specific
 * energy: rho := rho_Tr, p := rho_Tr v, E := rho_Tr (E / rho).
 * At most cap sinks are written (the cells beyond are left as they are);
 * returns the number of cells that satisfy the conditions. */
int64_t or_create_sinks(const or_params *P, or_mesh *S, const or_mesh *B, int64_t cap, double *x, double *y,
                        double *z, double *m, double *px, double *py, double *pz)
{
    if (!P || !S || !B || P->kind != KIND_SINK) return -1;
    int nx = S->n[0], ny = S->n[1], nz = S->n[2];
    int R = stencil_halfwidth(P->r_K);
    double r2 = P->r_K * P->r_K;
    double V = cell_volume(S->dx);
    int64_t nvalid = (int64_t)nx * ny * nz;
    unsigned char *flag = (unsigned char *)calloc((size_t)(nvalid > 0 ? nvalid : 1), 1);
    if (!flag) return -1;
    int64_t v = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++, v++) {
                double U[NF], D[NF], cs, rtr;
                read_state(S, i, j, k, U);
                int64_t b = cell_index(B, i, j, k);
                for (int f = 0; f < NF; f++) D[f] = B->u[(int64_t)f * B->fstride + b];
                if (!all_zero(D)) continue;                       /* (c) */
                sink_cell(P, S->dx, U, &cs, &rtr);
                if (!(U[0] > rtr)) continue;                      /* (a) */
                int ok = 1;
                for (int oz = -R; oz <= R && ok; oz++)
                    for (int oy = -R; oy <= R && ok; oy++)
                        for (int ox = -R; ox <= R && ok; ox++) {
                            if (!ox && !oy && !oz) continue;
                            double d2 = (double)(ox * ox + oy * oy) + (double)(oz * oz);
                            if (!(d2 < r2)) continue;
                            int a = i + ox, bb = j + oy, c = k + oz;
                            if (a < 0 || a >= nx) { if (!S->periodic[0]) continue; a = (a + nx) % nx; }
                            if (bb < 0 || bb >= ny) { if (!S->periodic[1]) continue; bb = (bb + ny) % ny; }
                            if (c < 0 || c >= nz) { if (!S->periodic[2]) continue; c = (c + nz) % nz; }
                            if (a == i && bb == j && c == k) continue; /* a small periodic box wraps onto c */
                            double rho2 = S->u[cell_index(S, a, bb, c)];
                            if (!(U[0] > rho2)) ok = 0;          /* (b) */
                        }
                flag[v] = (unsigned char)ok;
            }
    int64_t n = 0;
    v = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++, v++) {
                if (!flag[v]) continue;
                if (n < cap) {
                    double U[NF], cs, rtr;
                    read_state(S, i, j, k, U);
                    sink_cell(P, S->dx, U, &cs, &rtr);
                    double vel[3] = {U[1] / U[0], U[2] / U[0], U[3] / U[0]};
                    double es = U[4] / U[0];
                    double ms = (U[0] - rtr) * V;
                    x[n] = (double)i + 0.5;
                    y[n] = (double)j + 0.5;
                    z[n] = (double)k + 0.5;
                    m[n] = ms;
                    px[n] = ms * vel[0];
                    py[n] = ms * vel[1];
                    pz[n] = ms * vel[2];
                    int64_t c = cell_index(S, i, j, k);
                    S->u[c] = rtr;
                    for (int a = 0; a < 3; a++) S->u[(int64_t)(1 + a) * S->fstride + c] = rtr * vel[a];
                    S->u[(int64_t)4 * S->fstride + c] = rtr * es;
                }
                n++;
            }
    free(flag);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Sampled evaluation for large boxes: cells and particles one by one        */
/* ------------------------------------------------------------------------ */

/* Particles binned by host cell (a stable counting sort: within a bin the
 * particle indices ascend).  Pure bookkeeping, no arithmetic of the method. */
typedef struct {
    int64_t ncell;
    int64_t *start; /* [ncell + 1] */
    int64_t *idx;   /* [count] */
} or_bins;

static int64_t host_key(const or_mesh *S, double x, double y, double z)
{
    int64_t hx = (int64_t)floor(x), hy = (int64_t)floor(y), hz = (int64_t)floor(z);
    return (hz * S->n[1] + hy) * S->n[0] + hx;
}

or_bins *or_bins_build(const or_mesh *S, const or_particles *p)
{
    or_bins *b = (or_bins *)calloc(1, sizeof(or_bins));
    if (!b) return NULL;
    b->ncell = (int64_t)S->n[0] * S->n[1] * S->n[2];
    b->start = (int64_t *)calloc((size_t)b->ncell + 1, sizeof(int64_t));
    b->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p->count > 0 ? p->count : 1));
    if (!b->start || !b->idx) { free(b->start); free(b->idx); free(b); return NULL; }
    for (int64_t s = 0; s < p->count; s++) {
        if (check_position(S, p->x[s], p->y[s], p->z[s])) continue;
        b->start[host_key(S, p->x[s], p->y[s], p->z[s]) + 1]++;
    }
    for (int64_t c = 0; c < b->ncell; c++) b->start[c + 1] += b->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)b->ncell);
    if (!fill) { free(b->start); free(b->idx); free(b); return NULL; }
    memcpy(fill, b->start, sizeof(int64_t) * (size_t)b->ncell);
    for (int64_t s = 0; s < p->count; s++) {
        if (check_position(S, p->x[s], p->y[s], p->z[s])) continue;
        b->idx[fill[host_key(S, p->x[s], p->y[s], p->z[s])]++] = s;
    }
    free(fill);
    return b;
}

void or_bins_free(or_bins *b)
{
    if (!b) return;
    free(b->start);
    free(b->idx);
    free(b);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : x > y;
}

/* Particles whose (unwrapped) kernel can reach buffer coordinate (bi, bj, bk),
 * in ascending index order.  Returns the count; *out is malloc'ed. */
static int64_t candidates(const or_mesh *S, const or_bins *bins, int R, int bi, int bj, int bk, int64_t **out)
{
    int lo[3], hi[3], b[3] = {bi, bj, bk};
    for (int a = 0; a < 3; a++) {
        lo[a] = b[a] - R < 0 ? 0 : b[a] - R;
        hi[a] = b[a] + R > S->n[a] - 1 ? S->n[a] - 1 : b[a] + R;
    }
    int64_t n = 0;
    for (int k = lo[2]; k <= hi[2]; k++)
        for (int j = lo[1]; j <= hi[1]; j++)
            for (int i = lo[0]; i <= hi[0]; i++) {
                int64_t c = ((int64_t)k * S->n[1] + j) * S->n[0] + i;
                n += bins->start[c + 1] - bins->start[c];
            }
    int64_t *v = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t t = 0;
    for (int k = lo[2]; k <= hi[2]; k++)
        for (int j = lo[1]; j <= hi[1]; j++)
            for (int i = lo[0]; i <= hi[0]; i++) {
                int64_t c = ((int64_t)k * S->n[1] + j) * S->n[0] + i;
                for (int64_t q = bins->start[c]; q < bins->start[c + 1]; q++) v[t++] = bins->idx[q];
            }
    qsort(v, (size_t)n, sizeof(int64_t), cmp_i64);
    *out = v;
    return n;
}

/* Step-1 buffer value at one unwrapped buffer coordinate: the same sum as
 * or_deposit restricted to that cell (same particle order, same values). */
static int deposit_at(const or_params *P, const or_mesh *S, const or_particles *p, const or_bins *bins, kcell *kc,
                      int bi, int bj, int bk, double out[NF], double absout[NF])
{
    int R = stencil_halfwidth(P->r_K);
    int64_t *cand;
    int64_t nc = candidates(S, bins, R, bi, bj, bk, &cand);
    double G[MAX_ROWS];
    int status = OR_OK;
    for (int f = 0; f < NF; f++) { out[f] = 0.0; absout[f] = 0.0; }
    for (int64_t t = 0; t < nc; t++) {
        int64_t s = cand[t];
        double x = p->x[s], y = p->y[s], z = p->z[s];
        int nk = kernel_cells(S, P->r_K, x, y, z, kc);
        int hit = -1;
        for (int q = 0; q < nk; q++)
            if (kc[q].ci == bi && kc[q].cj == bj && kc[q].ck == bk) { hit = q; break; }
        if (hit < 0) continue;
        kcell c = kc[hit];
        int st = gather_one(P, S, p, s, kc, G, 1);
        if (st && !status) status = st;
        double w = cell_fraction(P, &c, x, y, z);
        if (w == 0.0) continue;
        double U[NF], dU[NF];
        read_state(S, c.wi, c.wj, c.wk, U);
        kind_delta(P, S->dx, w, U, G, 1, &c, dU);
        for (int f = 0; f < NF; f++) { out[f] = out[f] + dU[f]; absout[f] = absout[f] + fabs(dU[f]); }
    }
    free(cand);
    return status;
}

/* Step-2 (summed) buffer value at a valid cell, images in the or_fold order. */
static int folded_at(const or_params *P, const or_mesh *S, const or_particles *p, const or_bins *bins, int g,
                     kcell *kc, int i, int j, int k, double out[NF], double absout[NF])
{
    int status = deposit_at(P, S, p, bins, kc, i, j, k, out, absout);
    int nx = S->n[0], ny = S->n[1], nz = S->n[2];
    for (int oz = -1; oz <= 1; oz++)
        for (int oy = -1; oy <= 1; oy++)
            for (int ox = -1; ox <= 1; ox++) {
                if (ox == 0 && oy == 0 && oz == 0) continue;
                if ((ox && !S->periodic[0]) || (oy && !S->periodic[1]) || (oz && !S->periodic[2])) continue;
                int gi = i + ox * nx, gj = j + oy * ny, gk = k + oz * nz;
                if (gi < -g || gi >= nx + g || gj < -g || gj >= ny + g || gk < -g || gk >= nz + g) continue;
                double v[NF], av[NF];
                int st = deposit_at(P, S, p, bins, kc, gi, gj, gk, v, av);
                if (st && !status) status = st;
                for (int f = 0; f < NF; f++) { out[f] = out[f] + v[f]; absout[f] = absout[f] + av[f]; }
            }
    return status;
}

/* For each listed valid cell (ijk triplets): the summed buffer (out_sum,
 * [ncells][5]), its |.| analogue (out_abs) and the updated state (out_new). */
int or_cells_at(const or_params *P, const or_mesh *S, const or_particles *p, const or_bins *bins, int g,
                int64_t ncells, const int32_t *ijk, double *out_sum, double *out_abs, double *out_new, double *out_eta)
{
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return OR_ERR_NOMEM;
    int status = OR_OK;
    for (int64_t t = 0; t < ncells; t++) {
        int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
        double D[NF], A[NF], U[NF];
        int st = folded_at(P, S, p, bins, g, kc, i, j, k, D, A);
        if (st && !status) status = st;
        read_state(S, i, j, k, U);
        double eta[NF];
        int nr;
        kind_eta(P, S->dx, U, D, eta, &nr);
        int zero = all_zero(D);
        for (int f = 0; f < NF; f++) {
            out_sum[NF * t + f] = D[f];
            out_abs[NF * t + f] = A[f];
            out_new[NF * t + f] = zero ? U[f] : U[f] + eta[f] * D[f];
        }
        if (out_eta) out_eta[t] = eta[1];
    }
    free(kc);
    return status;
}

/* Step 4 for listed sinks only: updated (m, px, py, pz) into out [n][4]. */
int or_sinks_at(const or_params *P, const or_mesh *S, const or_particles *p, const or_bins *bins, int g,
                int64_t nsel, const int64_t *sel, double *out)
{
    if (P->kind != KIND_SINK) return OR_ERR_ARG;
    kcell *kc = alloc_kcells(P->r_K);
    kcell *kc2 = alloc_kcells(P->r_K);
    if (!kc || !kc2) { free(kc); free(kc2); return OR_ERR_NOMEM; }
    double V = cell_volume(S->dx);
    double G[SK_ROWS];
    int status = OR_OK;
    for (int64_t t = 0; t < nsel; t++) {
        int64_t s = sel[t];
        int st = gather_sink_one(P, S, p, s, kc, G, 1);
        if (st && !status) status = st;
        int nk = kernel_cells(S, P->r_K, p->x[s], p->y[s], p->z[s], kc);
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = 0; q < nk; q++) {
            double U[NF], dU[NF], D[NF], A[NF];
            read_state(S, kc[q].wi, kc[q].wj, kc[q].wk, U);
            sink_delta(P, S->dx, U, G, 1, &kc[q], dU);
            st = folded_at(P, S, p, bins, g, kc2, kc[q].wi, kc[q].wj, kc[q].wk, D, A);
            if (st && !status) status = st;
            double eta = sink_eta(P, S->dx, U, D);
            return_add(eta, U, dU, acc);
        }
        out[4 * t + 0] = p->m[s] - acc[0] * V;
        out[4 * t + 1] = p->px[s] - acc[1] * V;
        out[4 * t + 2] = p->py[s] - acc[2] * V;
        out[4 * t + 3] = p->pz[s] - acc[3] * V;
    }
    free(kc);
    free(kc2);
    return status;
}

/* Gathered rows of listed particles only ([rows][nsel]). */
int or_gather_at(const or_params *P, const or_mesh *S, const or_particles *p, int64_t nsel, const int64_t *sel,
                 double *gathered)
{
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return OR_ERR_NOMEM;
    int status = OR_OK;
    for (int64_t t = 0; t < nsel; t++) {
        int st = gather_one(P, S, p, sel[t], kc, gathered + t, nsel);
        if (st && !status) status = st;
    }
    free(kc);
    return status;
}

/* Kernel cells of one particle (for tests): unwrapped ijk, omega; returns n. */
int or_kernel_of(const or_params *P, const or_mesh *S, double x, double y, double z, int32_t *ijk, double *omega)
{
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return -1;
    int nk = kernel_cells(S, P->r_K, x, y, z, kc);
    for (int t = 0; t < nk; t++) {
        ijk[3 * t] = kc[t].ci;
        ijk[3 * t + 1] = kc[t].cj;
        ijk[3 * t + 2] = kc[t].ck;
        omega[t] = cell_fraction(P, &kc[t], x, y, z);
    }
    free(kc);
    return nk;
}

/* Deposition function of ONE particle: its kernel cells (unwrapped ijk) and
 * Delta U^s_c ([n][5]) from its gathered row G ([rows][1]); returns n.  Used
 * by the finite-difference tests of the adjoint. */
int or_deltas(const or_params *P, const or_mesh *S, const or_particles *p, const double *G, int32_t *ijk, double *dU)
{
    kcell *kc = alloc_kcells(P->r_K);
    if (!kc) return -1;
    double x = p->x[0], y = p->y[0], z = p->z[0];
    int nk = kernel_cells(S, P->r_K, x, y, z, kc);
    int n = 0;
    for (int t = 0; t < nk; t++) {
        double w = cell_fraction(P, &kc[t], x, y, z);
        if (w == 0.0) continue;
        double U[NF], d[NF];
        read_state(S, kc[t].wi, kc[t].wj, kc[t].wk, U);
        kind_delta(P, S->dx, w, U, G, 1, &kc[t], d);
        ijk[3 * n] = kc[t].ci;
        ijk[3 * n + 1] = kc[t].cj;
        ijk[3 * n + 2] = kc[t].ck;
        for (int f = 0; f < NF; f++) dU[NF * n + f] = d[f];
        n++;
    }
    free(kc);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Batched form: many uneven patches of one level tiling a periodic domain   */
/* ------------------------------------------------------------------------ */

/* The patches form a rectilinear grid: every patch in a row of the grid has
 * the same extent across that row.  Patch p lists its neighbours in nb[p][26],
 * the patch displaced by o = (ox, oy, oz) in {-1,0,1}^3 \ {0}, in the order oz
 * slowest, ox fastest.  A padded coordinate c of patch p is then the valid
 * cell, on each axis a,
 *   c_a + n_q,a   of the neighbour q below   (c_a < 0),
 *   c_a - n_p,a   of the neighbour q above   (c_a >= n_p,a),
 *   c_a           otherwise,
 * q being nb[p][o] with o_a the sign of the case.  Each patch keeps state
 * and buffer at offset[p] of two arenas, [5][fstride[p]], padded by ng ghost
 * cells; its particles are [first[p], first[p] + count[p]) of one particle
 * set, in patch-local cell units, and their gathered rows have stride
 * first[np] (the total count). */
typedef struct {
    int32_t np;             /* number of patches */
    int32_t ng;             /* ghost cells per side, the same for every patch */
    double dx;              /* cell size (one level) */
    const int32_t *dims;    /* [np][3] valid cells per axis */
    const int32_t *nb;      /* [np][26] neighbour patches */
    const int64_t *offset;  /* [np] arena offset of (field 0, padded cell 0) */
    const int64_t *fstride; /* [np] elements between fields */
    const int64_t *first;   /* [np + 1] particle ranges, first[np] = total */
} or_batch;

static int nb_slot(int ox, int oy, int oz)
{
    int t = ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1);
    return t > 13 ? t - 1 : t;
}

static or_mesh batch_view(const or_batch *T, int p, double *arena)
{
    or_mesh M;
    for (int a = 0; a < 3; a++) { M.n[a] = T->dims[3 * p + a]; M.periodic[a] = 2; }
    M.ng = T->ng;
    M.pad_ = 0;
    M.dx = T->dx;
    M.fstride = T->fstride[p];
    M.u = arena + T->offset[p];
    return M;
}

/* Owning (patch, valid coordinate) of padded coordinate c of patch p. */
static int batch_owner(const or_batch *T, int p, const int c[3], int w[3])
{
    const int32_t *np_ = T->dims + 3 * p;
    int o[3];
    for (int a = 0; a < 3; a++) o[a] = c[a] < 0 ? -1 : (c[a] >= np_[a] ? 1 : 0);
    int q = (o[0] || o[1] || o[2]) ? T->nb[26 * p + nb_slot(o[0], o[1], o[2])] : p;
    for (int a = 0; a < 3; a++) w[a] = c[a] + (o[a] < 0 ? T->dims[3 * q + a] : 0) - (o[a] > 0 ? np_[a] : 0);
    return q;
}

/* Every ghost cell of the first `owned` patches := the cell it stands for
 * (all 5 fields). */
static void batch_fill_ghosts_n(const or_batch *T, int owned, double *arena)
{
    int g = T->ng;
    for (int p = 0; p < owned; p++) {
        or_mesh M = batch_view(T, p, arena);
        for (int k = -g; k < M.n[2] + g; k++)
            for (int j = -g; j < M.n[1] + g; j++)
                for (int i = -g; i < M.n[0] + g; i++) {
                    if (i >= 0 && i < M.n[0] && j >= 0 && j < M.n[1] && k >= 0 && k < M.n[2]) continue;
                    int c[3] = {i, j, k}, w[3];
                    int q = batch_owner(T, p, c, w);
                    or_mesh Q = batch_view(T, q, arena);
                    int64_t src = cell_index(&Q, w[0], w[1], w[2]), dst = cell_index(&M, i, j, k);
                    for (int f = 0; f < NF; f++) M.u[(int64_t)f * M.fstride + dst] = Q.u[(int64_t)f * Q.fstride + src];
                }
    }
}

/* Ghost-zone summation across patches (Step 2, App. A.2): each valid cell c of
 * patch p becomes ((B_c + B_img1) + B_img2) + ... over its ghost images, taken
 * in lexicographic order of the image offset (oz, oy, ox).  The image at
 * offset o lies in the patch q = nb[p][-o], at c_a + n_q,a (o_a = 1),
 * c_a - n_p,a (o_a = -1) or c_a (o_a = 0), when that is inside q's padded
 * box.  With one patch whose neighbours are all itself this is the fold of a
 * periodic box.  Ghost cells are only read, so the fold runs in place. */
static void batch_fold_arena_n(const or_batch *T, int owned, double *arena)
{
    int g = T->ng;
    for (int p = 0; p < owned; p++) {
        or_mesh M = batch_view(T, p, arena);
        for (int f = 0; f < NF; f++)
            for (int k = 0; k < M.n[2]; k++)
                for (int j = 0; j < M.n[1]; j++)
                    for (int i = 0; i < M.n[0]; i++) {
                        int64_t c = cell_index(&M, i, j, k);
                        double v = M.u[(int64_t)f * M.fstride + c];
                        for (int oz = -1; oz <= 1; oz++)
                            for (int oy = -1; oy <= 1; oy++)
                                for (int ox = -1; ox <= 1; ox++) {
                                    if (ox == 0 && oy == 0 && oz == 0) continue;
                                    int q = T->nb[26 * p + nb_slot(-ox, -oy, -oz)];
                                    int o[3] = {ox, oy, oz}, cc[3] = {i, j, k}, gi[3], in = 1;
                                    for (int a = 0; a < 3; a++) {
                                        int nq = T->dims[3 * q + a], npa = M.n[a];
                                        gi[a] = cc[a] + (o[a] > 0 ? nq : 0) - (o[a] < 0 ? npa : 0);
                                        if (gi[a] < -g || gi[a] >= nq + g) in = 0;
                                    }
                                    if (!in) continue;
                                    or_mesh Q = batch_view(T, q, arena);
                                    v = v + Q.u[(int64_t)f * Q.fstride + cell_index(&Q, gi[0], gi[1], gi[2])];
                                }
                        M.u[(int64_t)f * M.fstride + c] = v;
                    }
    }
}

static void batch_fill_ghosts(const or_batch *T, double *arena) { batch_fill_ghosts_n(T, T->np, arena); }
static void batch_fold_arena(const or_batch *T, double *arena) { batch_fold_arena_n(T, T->np, arena); }

static int64_t batch_arena_len(const or_batch *T)
{
    int64_t len = 0;
    for (int p = 0; p < T->np; p++) {
        int64_t e = T->offset[p] + (int64_t)NF * T->fstride[p];
        if (e > len) len = e;
    }
    return len;
}

static int batch_check(const or_params *P, const or_batch *T)
{
    if (!T || T->np <= 0 || T->ng < stencil_halfwidth(P->r_K) || P->kind == KIND_MASS) return OR_ERR_ARG;
    for (int p = 0; p < T->np; p++)
        for (int a = 0; a < 3; a++)
            if (T->dims[3 * p + a] < T->ng) return OR_ERR_ARG;
    return OR_OK;
}

/* Exported for tests: fills the ghosts of a state arena, or folds a buffer
 * arena, with the rules above. */
void or_batch_fill_ghosts(const or_batch *T, double *arena) { batch_fill_ghosts(T, arena); }
void or_batch_fold(const or_batch *T, double *arena) { batch_fold_arena(T, arena); }

/* A private copy of the state whose first `owned` patches have their ghost
 * cells filled from the cells they stand for (the caller's ghost cells are
 * never read). */
static double *batch_state_scratch(const or_batch *T, int owned, const double *state)
{
    int64_t len = batch_arena_len(T);
    double *scratch = (double *)malloc(sizeof(double) * (size_t)len);
    if (!scratch) return NULL;
    memcpy(scratch, state, sizeof(double) * (size_t)len);
    batch_fill_ghosts_n(T, owned, scratch);
    return scratch;
}

/* First part of a pass over the first `owned` patches of a batch (Step 1):
 * their buffers (and absbuf) zeroed, ghosts included, then the particles of
 * patch 0, 1, ... each in index order gathered and deposited.  The other
 * patches of the batch are only read, as neighbours (they stand for patches
 * that another rank owns: their valid state cells must hold what those
 * patches hold). */
static int batch_part_deposit(const or_params *P, const or_batch *T, int owned, const double *state, double *buf,
                              double *absbuf, or_particles *p, double *gathered)
{
    double *scratch = batch_state_scratch(T, owned, state);
    kcell *kc = alloc_kcells(P->r_K);
    if (!scratch || !kc) { free(scratch); free(kc); return OR_ERR_NOMEM; }
    for (int q = 0; q < owned; q++) {
        or_mesh B = batch_view(T, q, buf);
        int64_t pc = (int64_t)(B.n[0] + 2 * B.ng) * (B.n[1] + 2 * B.ng) * (B.n[2] + 2 * B.ng);
        for (int f = 0; f < NF; f++)
            for (int64_t c = 0; c < pc; c++) {
                B.u[(int64_t)f * B.fstride + c] = 0.0;
                if (absbuf) absbuf[T->offset[q] + (int64_t)f * B.fstride + c] = 0.0;
            }
    }
    int status = OR_OK;
    int64_t N = T->first[T->np];
    for (int q = 0; q < owned && !status; q++) {
        or_mesh S = batch_view(T, q, scratch), B = batch_view(T, q, buf);
        int64_t f0 = T->first[q];
        or_particles pp = {T->first[q + 1] - f0, p->x + f0, p->y + f0, p->z + f0,
                           p->m + f0, p->px + f0, p->py + f0, p->pz + f0, p->e ? p->e + f0 : NULL};
        for (int64_t s = 0; s < pp.count; s++) {
            int r = P->kind == KIND_FEEDBACK ? gather_feedback_one(P, &S, &pp, s, kc, gathered + f0 + s, N)
                                             : gather_sink_one(P, &S, &pp, s, kc, gathered + f0 + s, N);
            if (r && !status) status = r;
        }
        if (status) break;
        int r = deposit_parts(P, &S, &pp, gathered + f0, N, &B, absbuf ? absbuf + T->offset[q] : NULL);
        if (r && !status) status = r;
    }
    free(scratch);
    free(kc);
    return status;
}

/* Second part (Steps 2-5) over the first `owned` patches: the cross-patch
 * fold of their buffers (images read from every neighbour's ghost cells),
 * for sinks Step 4 with eta at a ghost image taken from the cell it stands
 * for (a neighbour that stands for another rank's patch must hold that
 * patch's folded sums in its valid buffer cells), and the limited update of
 * their valid cells.  eta_out: one value per valid cell of those patches. */
static int batch_part_finish(const or_params *P, const or_batch *T, int owned, double *state, double *buf,
                             double *absbuf, or_particles *p, const double *gathered, double *eta_out, int64_t *counts)
{
    int status = OR_OK;
    int64_t len = batch_arena_len(T), N = T->first[T->np];
    batch_fold_arena_n(T, owned, buf);
    if (absbuf) batch_fold_arena_n(T, owned, absbuf);
    if (P->kind == KIND_SINK) {
        double *scratch = batch_state_scratch(T, owned, state);
        double *bcopy = (double *)malloc(sizeof(double) * (size_t)len);
        if (!scratch || !bcopy) status = OR_ERR_NOMEM;
        else {
            memcpy(bcopy, buf, sizeof(double) * (size_t)len);
            batch_fill_ghosts_n(T, owned, bcopy);
            for (int q = 0; q < owned && !status; q++) {
                or_mesh S = batch_view(T, q, scratch), B = batch_view(T, q, bcopy);
                int64_t f0 = T->first[q];
                or_particles pp = {T->first[q + 1] - f0, p->x + f0, p->y + f0, p->z + f0,
                                   p->m + f0, p->px + f0, p->py + f0, p->pz + f0, NULL};
                status = return_parts(P, &S, &B, &pp, gathered + f0, N);
            }
        }
        free(scratch);
        free(bcopy);
    }
    if (!status) {
        int64_t tot[2] = {0, 0}, v = 0;
        for (int q = 0; q < owned; q++) {
            or_mesh S = batch_view(T, q, state), B = batch_view(T, q, buf);
            int64_t c2[2];
            or_apply(P, &S, &B, eta_out ? eta_out + v : NULL, c2);
            tot[0] += c2[0];
            tot[1] += c2[1];
            v += (int64_t)S.n[0] * S.n[1] * S.n[2];
        }
        if (counts) { counts[0] = tot[0]; counts[1] = tot[1]; }
    }
    return status;
}

/* One PMP pass (Sec. 2.2) over a batch: Steps 1-5 with every patch's ghost
 * cells read through its neighbours, particles of patch 0, 1, ... each in
 * index order, the cross-patch fold above, Step 4 with eta at a ghost image
 * taken from the cell it stands for, and the limited update of every valid
 * cell.  buf (and absbuf) receive the deposits including ghosts, then the
 * folded sums in valid cells.  eta_out gets one value per valid cell, patch
 * after patch (x fastest).  counts as for or_apply, summed. */
int or_batch_cycle(const or_params *P, const or_batch *T, double *state, double *buf, double *absbuf,
                   or_particles *p, double *gathered, double *eta_out, int64_t *counts)
{
    int st = batch_check(P, T);
    if (st) return st;
    if (!p || !gathered || !state || !buf || p->count != T->first[T->np]) return OR_ERR_ARG;
    st = batch_part_deposit(P, T, T->np, state, buf, absbuf, p, gathered);
    if (!st) st = batch_part_finish(P, T, T->np, state, buf, absbuf, p, gathered, eta_out, counts);
    return st;
}

/* The two parts of a pass over the first `owned` patches of a batch, for a
 * rank of a decomposition whose other patches stand for neighbours owned
 * elsewhere: part 0 is Step 1 (gather and deposit), part 1 Steps 2-5.
 * Between them the caller brings in the ghost cells of those neighbours'
 * buffers (their deposits that fall on owned cells) and, for sinks, their
 * folded sums; before part 0 their valid state cells.  Run on one rank that
 * owns every patch, part 0 then part 1 is or_batch_cycle. */
int or_batch_part(const or_params *P, const or_batch *T, int32_t owned, int32_t part, double *state, double *buf,
                  or_particles *p, double *gathered, double *eta_out, int64_t *counts)
{
    int st = batch_check(P, T);
    if (st) return st;
    if (!p || !gathered || !state || !buf || p->count != T->first[T->np] || owned < 0 || owned > T->np)
        return OR_ERR_ARG;
    if (part == 0) return batch_part_deposit(P, T, owned, state, buf, NULL, p, gathered);
    if (part == 1) return batch_part_finish(P, T, owned, state, buf, NULL, p, gathered, eta_out, counts);
    return OR_ERR_ARG;
}
