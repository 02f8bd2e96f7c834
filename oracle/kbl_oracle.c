/*
 * kbl_oracle.c -- FP64 CPU oracle of the kinetic-bounds limiter (arXiv
 * 2407.20966) and of the nodal DG / FR Euler stage it sits in.
 *
 * TEST INFRASTRUCTURE ONLY: plain loops in the paper's order, no blocking, no
 * fusion, no reordering beyond what the definitions state.  It shares no code
 * with the CUDA library.  Conventions are in kbl_oracle.h.
 */
#include "kbl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

int orc_nv(const orc_cfg* c) { return c->dim + 2; }
int orc_ns(const orc_cfg* c) { return c->dim == 1 ? c->p + 1 : (c->p + 1) * (c->p + 1); }
int orc_nfp(const orc_cfg* c) { return c->dim == 1 ? 2 : 4 * (c->p + 1); }
int orc_nstencil(const orc_cfg* c) { return c->stencil == 1 ? 3 * orc_ns(c) : orc_ns(c) + 2 * orc_nfp(c); }
static int nfp_face(const orc_cfg* c) { return c->dim == 1 ? 1 : c->p + 1; }

/* ===================================================================== */
/* One-dimensional polynomial tools                                       */
/* ===================================================================== */

/* Legendre polynomial P_n and its derivative by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
void orc_legendre(int n, double x, double* P, double* dP)
{
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (n == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        double d2 = d0 + (2.0 * k + 1.0) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *P = p1; *dP = d1;
}

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1]: roots of P_n by
 * Newton's method, w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).  These are the
 * solution and flux points the paper uses for lines and quadrilaterals (Sec. 5). */
int orc_gauss_legendre(int n, double* x, double* w)
{
    if (n < 1) return -2;
    for (int i = 0; i < n; i++) {
        double r = -cos(ORC_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double P, dP;
            orc_legendre(n, r, &P, &dP);
            double dr = P / dP;
            r -= dr;
            if (fabs(dr) < 1e-16) break;
        }
        double P, dP;
        orc_legendre(n, r, &P, &dP);
        x[i] = r;
        w[i] = 2.0 / ((1.0 - r * r) * dP * dP);
    }
    return 0;
}

/* Lagrange basis polynomial l_j of the nodes, evaluated at x. */
double orc_lagrange(int n, const double* nodes, int j, double x)
{
    double v = 1.0;
    for (int m = 0; m < n; m++)
        if (m != j) v *= (x - nodes[m]) / (nodes[j] - nodes[m]);
    return v;
}

/* Derivative of l_j at x: sum over l != j of 1/(x_j - x_l) times the product
 * of the remaining factors. */
double orc_lagrange_deriv(int n, const double* nodes, int j, double x)
{
    double s = 0.0;
    for (int l = 0; l < n; l++) {
        if (l == j) continue;
        double t = 1.0 / (nodes[j] - nodes[l]);
        for (int m = 0; m < n; m++)
            if (m != j && m != l) t *= (x - nodes[m]) / (nodes[j] - nodes[m]);
        s += t;
    }
    return s;
}

/* Derivatives of the FR correction functions that recover nodal DG (Huynh's
 * g_DG, the right and left Radau polynomials of degree p+1):
 *   g_L = (-1)^(p+1)/2 (P_{p+1} - P_p),  g_L(-1) = 1, g_L(1) = 0,
 *   g_R = 1/2 (P_{p+1} + P_p),           g_R(-1) = 0, g_R(1) = 1. */
void orc_correction_deriv(int p, double x, double* dgl, double* dgr)
{
    double Pa, dPa, Pb, dPb;
    orc_legendre(p + 1, x, &Pa, &dPa);
    orc_legendre(p, x, &Pb, &dPb);
    double sgn = ((p + 1) % 2 == 0) ? 1.0 : -1.0;
    *dgl = 0.5 * sgn * (dPa - dPb);
    *dgr = 0.5 * (dPa + dPb);
}

/* ===================================================================== */
/* Euler physics                                                          */
/* ===================================================================== */

/* Ideal-gas pressure P = (gamma - 1)(E - m.m / (2 rho)), Eq. 3. */
double orc_pressure(const orc_cfg* c, const double* w)
{
    int d = c->dim;
    double mm = 0.0;
    for (int k = 0; k < d; k++) mm += w[1 + k] * w[1 + k];
    return (c->gamma - 1.0) * (w[d + 1] - 0.5 * mm / w[0]);
}

/* Physical flux along axis `dir`, Eq. 2: [m_dir, m U_dir + P e_dir, (E + P) U_dir]. */
void orc_flux(const orc_cfg* c, const double* w, int dir, double* F)
{
    int d = c->dim;
    double P = orc_pressure(c, w);
    double U = w[1 + dir] / w[0];
    F[0] = w[1 + dir];
    for (int k = 0; k < d; k++) F[1 + k] = w[1 + k] * U + (k == dir ? P : 0.0);
    F[d + 1] = (w[d + 1] + P) * U;
}

/* Rusanov flux with the Davis wavespeed (assumption (iv) of Sec. 4 and its
 * remark): wl is on the minus side of the axis, wr on the plus side,
 *   F = 1/2 (F(wl) + F(wr)) - 1/2 lambda (wr - wl),
 *   lambda = max(|U_l| + c_l, |U_r| + c_r), c = sqrt(gamma P / rho). */
void orc_rusanov(const orc_cfg* c, const double* wl, const double* wr, int dir,
                 double* F)
{
    int nv = orc_nv(c);
    double Fl[4], Fr[4];
    orc_flux(c, wl, dir, Fl);
    orc_flux(c, wr, dir, Fr);
    double Pl = orc_pressure(c, wl), Pr = orc_pressure(c, wr);
    double sl = fabs(wl[1 + dir] / wl[0]) + sqrt(c->gamma * Pl / wl[0]);
    double sr = fabs(wr[1 + dir] / wr[0]) + sqrt(c->gamma * Pr / wr[0]);
    double lam = sl > sr ? sl : sr;
    for (int v = 0; v < nv; v++) F[v] = 0.5 * (Fl[v] + Fr[v]) - 0.5 * lam * (wr[v] - wl[v]);
}

/* HLLC flux (Toro, Spruce & Speares 1994, the Riemann solver of the paper's
 * experiments, Sec. 5) with the Davis wave-speed estimates
 *   S_l = min(U_l - c_l, U_r - c_r),  S_r = max(U_l + c_l, U_r + c_r)
 * (U the velocity along the axis) and the contact speed
 *   S* = (P_r - P_l + rho_l U_l (S_l - U_l) - rho_r U_r (S_r - U_r))
 *        / (rho_l (S_l - U_l) - rho_r (S_r - U_r)).
 * The flux is F(w_l) for 0 <= S_l, F(w_l) + S_l (w*_l - w_l) for S_l <= 0 <= S*,
 * F(w_r) + S_r (w*_r - w_r) for S* <= 0 <= S_r and F(w_r) for S_r <= 0, with the
 * star state of side K
 *   w*_K = rho_K (S_K - U_K)/(S_K - S*) [1, S* along the axis, the other velocity
 *          components of K, E_K/rho_K + (S* - U_K)(S* + P_K/(rho_K (S_K - U_K)))]. */
void orc_hllc(const orc_cfg* c, const double* wl, const double* wr, int dir, double* F)
{
    int d = c->dim, nv = orc_nv(c);
    double Pl = orc_pressure(c, wl), Pr = orc_pressure(c, wr);
    double Ul = wl[1 + dir] / wl[0], Ur = wr[1 + dir] / wr[0];
    double cl = sqrt(c->gamma * Pl / wl[0]), cr = sqrt(c->gamma * Pr / wr[0]);
    double Sl = Ul - cl < Ur - cr ? Ul - cl : Ur - cr;
    double Sr = Ul + cl > Ur + cr ? Ul + cl : Ur + cr;
    double Ss = (Pr - Pl + wl[0] * Ul * (Sl - Ul) - wr[0] * Ur * (Sr - Ur)) /
                (wl[0] * (Sl - Ul) - wr[0] * (Sr - Ur));
    if (0.0 <= Sl) {
        orc_flux(c, wl, dir, F);
        return;
    }
    if (Sr <= 0.0) {
        orc_flux(c, wr, dir, F);
        return;
    }
    const double* w = Ss >= 0.0 ? wl : wr;
    double S = Ss >= 0.0 ? Sl : Sr, U = Ss >= 0.0 ? Ul : Ur, P = Ss >= 0.0 ? Pl : Pr;
    orc_flux(c, w, dir, F);
    double f = w[0] * (S - U) / (S - Ss), ws[4];
    ws[0] = f;
    for (int k = 0; k < d; k++) ws[1 + k] = f * (k == dir ? Ss : w[1 + k] / w[0]);
    ws[d + 1] = f * (w[d + 1] / w[0] + (Ss - U) * (Ss + P / (w[0] * (S - U))));
    for (int v = 0; v < nv; v++) F[v] += S * (ws[v] - w[v]);
}

/* HLL flux (Harten, Lax & van Leer 1983; the Riemann solver of the Sedov run,
 * Sec. 6.6) with the same Davis estimates S_l, S_r as above:
 *   F(w_l) for 0 <= S_l,  F(w_r) for S_r <= 0, and otherwise the flux of the single
 *   intermediate state,  (S_r F(w_l) - S_l F(w_r) + S_l S_r (w_r - w_l)) / (S_r - S_l). */
void orc_hll(const orc_cfg* c, const double* wl, const double* wr, int dir, double* F)
{
    int nv = orc_nv(c);
    double Pl = orc_pressure(c, wl), Pr = orc_pressure(c, wr);
    double Ul = wl[1 + dir] / wl[0], Ur = wr[1 + dir] / wr[0];
    double cl = sqrt(c->gamma * Pl / wl[0]), cr = sqrt(c->gamma * Pr / wr[0]);
    double Sl = Ul - cl < Ur - cr ? Ul - cl : Ur - cr;
    double Sr = Ul + cl > Ur + cr ? Ul + cl : Ur + cr;
    if (0.0 <= Sl) {
        orc_flux(c, wl, dir, F);
        return;
    }
    if (Sr <= 0.0) {
        orc_flux(c, wr, dir, F);
        return;
    }
    double Fl[4], Fr[4];
    orc_flux(c, wl, dir, Fl);
    orc_flux(c, wr, dir, Fr);
    for (int v = 0; v < nv; v++) F[v] = (Sr * Fl[v] - Sl * Fr[v] + Sl * Sr * (wr[v] - wl[v])) / (Sr - Sl);
}

/* The common flux of the configuration: Rusanov (c->flux == 0), HLLC (1) or HLL (2). */
static void orc_common_flux(const orc_cfg* c, const double* wl, const double* wr, int dir, double* F)
{
    if (c->flux == 1) orc_hllc(c, wl, wr, dir, F);
    else if (c->flux == 2) orc_hll(c, wl, wr, dir, F);
    else orc_rusanov(c, wl, wr, dir, F);
}

/* ===================================================================== */
/* Kinetic bounds                                                          */
/* ===================================================================== */

typedef struct {
    double rho, U[2], theta, A, cI;
} orc_maxw;

/* Primitive state of a stencil node and the constants of its Maxwellian,
 * Eq. 8:  g(u) = rho (2 pi theta)^(-d/2) exp(-|u - U|^2 / (2 theta)),
 * theta = P / rho; and the internal-energy weight theta delta / 2 of Eq. 44,
 * delta = 2/(gamma - 1) - d. */
static int orc_maxwellian_of(const orc_cfg* c, const double* w, orc_maxw* g)
{
    int d = c->dim;
    double P = orc_pressure(c, w);
    if (!(w[0] > 0.0) || !(P > 0.0)) return -1;
    g->rho = w[0];
    for (int k = 0; k < d; k++) g->U[k] = w[1 + k] / w[0];
    g->theta = P / w[0];
    g->A = (d == 1) ? g->rho / sqrt(2.0 * ORC_PI * g->theta)
                    : g->rho / (2.0 * ORC_PI * g->theta);
    double delta = 2.0 / (c->gamma - 1.0) - d;
    g->cI = 0.5 * delta * g->theta;
    return 0;
}

static double orc_eval_maxwellian(int d, const orc_maxw* g, const double* u)
{
    double q = 0.0;
    for (int k = 0; k < d; k++) q += (u[k] - g->U[k]) * (u[k] - g->U[k]);
    return g->A * exp(-q / (2.0 * g->theta));
}

/* Truncated velocity domain, Eq. 45, read with the upper end at
 * max(U + k sqrt(theta)) (the printed "-" there is a sign slip: the text before
 * it describes U +- k sqrt(theta)).  Taken per dimension over the stencil. */
static void orc_box(int d, double kk, int nS, const orc_maxw* g, double* lo, double* hi)
{
    for (int k = 0; k < d; k++) {
        lo[k] = g[0].U[k] - kk * sqrt(g[0].theta);
        hi[k] = g[0].U[k] + kk * sqrt(g[0].theta);
        for (int i = 1; i < nS; i++) {
            double a = g[i].U[k] - kk * sqrt(g[i].theta);
            double b = g[i].U[k] + kk * sqrt(g[i].theta);
            if (a < lo[k]) lo[k] = a;
            if (b > hi[k]) hi[k] = b;
        }
    }
}

/* Romberg weight of node j, in units of h, on an axis of N equispaced nodes (the
 * quadrature Sec. 5 names beside the trapezoidal rule).  Romberg's method is linear in the
 * node values, so node j's weight is what the method returns for values 1 at node j and 0
 * elsewhere.  With N - 1 = 2^L m (m odd): R(k, 0) is the trapezoidal sum of step
 * 2^(L-k) h (k = 0 the coarsest), R(k, i) = R(k, i-1) + (R(k, i-1) - R(k-1, i-1)) / (4^i - 1)
 * for 1 <= i <= k, and the weight is R(L, L). */
double orc_romberg_weight(int N, int j)
{
    int L = 0;
    while ((N - 1) % (2 << L) == 0) L++;
    double R[24][24];
    for (int k = 0; k <= L; k++) {
        int step = 1 << (L - k);
        R[k][0] = (j % step != 0) ? 0.0 : (j == 0 || j == N - 1) ? 0.5 * step : (double)step;
    }
    double four_i = 1.0;
    for (int i = 1; i <= L; i++) {
        four_i *= 4.0;
        for (int k = i; k <= L; k++) R[k][i] = R[k][i - 1] + (R[k][i - 1] - R[k - 1][i - 1]) / (four_i - 1.0);
    }
    return R[L][L];
}

/* Equispaced velocity grid over [lo, hi] (Sec. 3.7): u_j = lo + j h, h = (hi - lo)/(N - 1),
 * with trapezoidal weights (h, h/2 at both ends; rule 0) or Romberg weights (rule 1). */
static void orc_grid(int N, int rule, double lo, double hi, double* u, double* wq)
{
    double h = (hi - lo) / (N - 1);
    for (int j = 0; j < N; j++) {
        u[j] = lo + j * h;
        if (rule == 1) wq[j] = orc_romberg_weight(N, j) * h;
        else wq[j] = (j == 0 || j == N - 1) ? 0.5 * h : h;
    }
}

/* Add one velocity node's contribution to the moment bounds.
 *   density  Eq. 33:  sum M f_min,            sum M f_max
 *   momentum Eq. 35/36, per component: f_max where u_i < 0 and f_min where
 *            u_i >= 0 for the lower bound, the other way round for the upper
 *   energy   Eq. 34 with the internal-energy term of Eq. 42/44:
 *            sum M (f_T 1/2 |u|^2 + f_I)
 * lo/hi receive nv values each. */
static void orc_accumulate(int d, double M, const double* u, double Tlo, double Thi,
                           double Ilo, double Ihi, double* lo, double* hi)
{
    int nv = d + 2;
    lo[0] += M * Tlo;
    hi[0] += M * Thi;
    double ke = 0.0;
    for (int k = 0; k < d; k++) {
        ke += 0.5 * u[k] * u[k];
        if (u[k] < 0.0) {
            lo[1 + k] += M * Thi * u[k];
            hi[1 + k] += M * Tlo * u[k];
        } else {
            lo[1 + k] += M * Tlo * u[k];
            hi[1 + k] += M * Thi * u[k];
        }
    }
    lo[nv - 1] += M * (Tlo * ke + Ilo);
    hi[nv - 1] += M * (Thi * ke + Ihi);
}

#define ORC_MAX_S 256
#define ORC_MAX_NU 65536

int orc_velocity_box(const orc_cfg* c, int nS, const double* S, double* lo, double* hi)
{
    int nv = orc_nv(c);
    if (nS < 1 || nS > ORC_MAX_S) return -2;
    orc_maxw g[ORC_MAX_S];
    for (int i = 0; i < nS; i++)
        if (orc_maxwellian_of(c, S + i * nv, &g[i])) return -1;
    orc_box(c->dim, c->k, nS, g, lo, hi);
    return 0;
}

/* Shared walk over the velocity grid of stencil S.  which == -1: the
 * envelopes of Eq. 32 (with the relaxation of Eq. 40) give the bounds;
 * which == -2 / -3: the plain moments of f_min / f_max as distributions;
 * which >= 0: the single Maxwellian of node `which`, in the same order, so
 * every result can be compared with the bounds term by term. */
static int orc_walk(const orc_cfg* c, int nS, const double* S, int which,
                    double* lo, double* hi)
{
    int d = c->dim, nv = orc_nv(c);
    if (nS < 1 || nS > ORC_MAX_S) return -2;
    int Nx = c->nu[0], Ny = d == 2 ? c->nu[1] : 1;
    if (Nx < 2 || Nx > ORC_MAX_NU || (d == 2 && (Ny < 2 || Ny > ORC_MAX_NU))) return -2;
    if (c->quadrature == 1 && ((Nx - 1) % 2 != 0 || (d == 2 && (Ny - 1) % 2 != 0))) return -2;
    orc_maxw g[ORC_MAX_S];
    for (int i = 0; i < nS; i++)
        if (orc_maxwellian_of(c, S + i * nv, &g[i])) return -1;
    double blo[2], bhi[2];
    orc_box(d, c->k, nS, g, blo, bhi);
    double* ux = malloc(sizeof(double) * Nx);
    double* wx = malloc(sizeof(double) * Nx);
    double* uy = malloc(sizeof(double) * Ny);
    double* wy = malloc(sizeof(double) * Ny);
    orc_grid(Nx, c->quadrature, blo[0], bhi[0], ux, wx);
    if (d == 2) orc_grid(Ny, c->quadrature, blo[1], bhi[1], uy, wy);
    else { uy[0] = 0.0; wy[0] = 1.0; }
    for (int v = 0; v < nv; v++) lo[v] = hi[v] = 0.0;
    double r = c->r_fac;
    for (int jy = 0; jy < Ny; jy++) {
        for (int jx = 0; jx < Nx; jx++) {
            double u[2] = {ux[jx], uy[jy]};
            double M = (d == 2) ? wx[jx] * wy[jy] : wx[jx];
            double Tlo, Thi, Ilo, Ihi;
            if (which < 0) {
                /* Eq. 32: pointwise minimum and maximum over the stencil of
                 * the translational part g and of the internal part
                 * (theta delta / 2) g, each with its own envelope. */
                Tlo = INFINITY; Thi = -INFINITY; Ilo = INFINITY; Ihi = -INFINITY;
                for (int i = 0; i < nS; i++) {
                    double gi = orc_eval_maxwellian(d, &g[i], u);
                    double ci = g[i].cI * gi;
                    if (gi < Tlo) Tlo = gi;
                    if (gi > Thi) Thi = gi;
                    if (ci < Ilo) Ilo = ci;
                    if (ci > Ihi) Ihi = ci;
                }
                /* Eq. 40: relax the envelopes by (1 -+ r_fac). */
                Tlo *= (1.0 - r); Ilo *= (1.0 - r);
                Thi *= (1.0 + r); Ihi *= (1.0 + r);
                /* which == -2 / -3: plain moments of f_min / f_max alone */
                if (which == -2) { Thi = Tlo; Ihi = Ilo; }
                if (which == -3) { Tlo = Thi; Ilo = Ihi; }
            } else {
                double gi = orc_eval_maxwellian(d, &g[which], u);
                Tlo = Thi = gi;
                Ilo = Ihi = g[which].cI * gi;
            }
            orc_accumulate(d, M, u, Tlo, Thi, Ilo, Ihi, lo, hi);
        }
    }
    free(ux); free(wx); free(uy); free(wy);
    return 0;
}

/* Bounds of Sec. 3.3 (Eq. 32-36, 40, 42-46) for one stencil, then the density
 * floor of Sec. 3.8: rho_min <- max(rho_min, rho_floor). */
int orc_bounds_stencil(const orc_cfg* c, int nS, const double* S, double* wmin,
                       double* wmax)
{
    int rc = orc_walk(c, nS, S, -1, wmin, wmax);
    if (rc) return rc;
    if (wmin[0] < c->rho_floor) wmin[0] = c->rho_floor;
    return 0;
}

int orc_envelope_moments(const orc_cfg* c, int nS, const double* S, int upper, double* mom)
{
    double hi[4];
    return orc_walk(c, nS, S, upper ? -3 : -2, mom, hi);
}

int orc_state_moments(const orc_cfg* c, int nS, const double* S, int which, double* mom)
{
    if (which < 0 || which >= nS) return -2;
    double hi[4];
    return orc_walk(c, nS, S, which, mom, hi);
}

/* ===================================================================== */
/* Mesh-level operations                                                  */
/* ===================================================================== */

typedef struct {
    int n, ns, nfp, nfpf, nv;
    double x[16], wq[16];
    double lm[16], lp[16];      /* l_i(-1), l_i(+1) */
    double D[16][16];           /* D[i][m] = l_m'(x_i) */
    double gl[16], gr[16];      /* g_L'(x_i), g_R'(x_i) */
} orc_ops;

static void orc_build_ops(const orc_cfg* c, orc_ops* o)
{
    int n = c->p + 1;
    o->n = n;
    o->ns = orc_ns(c);
    o->nfp = orc_nfp(c);
    o->nfpf = nfp_face(c);
    o->nv = orc_nv(c);
    orc_gauss_legendre(n, o->x, o->wq);
    for (int i = 0; i < n; i++) {
        o->lm[i] = orc_lagrange(n, o->x, i, -1.0);
        o->lp[i] = orc_lagrange(n, o->x, i, 1.0);
        orc_correction_deriv(c->p, o->x[i], &o->gl[i], &o->gr[i]);
        for (int m = 0; m < n; m++) o->D[i][m] = orc_lagrange_deriv(n, o->x, m, o->x[i]);
    }
}

/* Interior values at the face points (interpolation of the element's
 * polynomial), in the face-point order of kbl_oracle.h. */
void orc_traces(const orc_cfg* c, const orc_mesh* m, const double* w, double* wf)
{
    orc_ops o;
    orc_build_ops(c, &o);
    int E = m->n_elem, n = o.n;
    for (int v = 0; v < o.nv; v++) {
        for (int e = 0; e < E; e++) {
            const double* we = w + ((size_t)v * E + e) * o.ns;
            double* fe = wf + ((size_t)v * E + e) * o.nfp;
            if (c->dim == 1) {
                double a = 0.0, b = 0.0;
                for (int i = 0; i < n; i++) { a += o.lm[i] * we[i]; b += o.lp[i] * we[i]; }
                fe[0] = a; fe[1] = b;
            } else {
                for (int k = 0; k < n; k++) {
                    double f0 = 0, f1 = 0, f2 = 0, f3 = 0;
                    for (int i = 0; i < n; i++) {
                        f0 += o.lm[i] * we[k * n + i];
                        f1 += o.lp[i] * we[k * n + i];
                        f2 += o.lm[i] * we[i * n + k];
                        f3 += o.lp[i] * we[i * n + k];
                    }
                    fe[0 * n + k] = f0; fe[1 * n + k] = f1;
                    fe[2 * n + k] = f2; fe[3 * n + k] = f3;
                }
            }
        }
    }
}

/* Exterior value at face point fp of element e: the neighbour's interior
 * value at the matching point, or the prescribed boundary state. */
static void orc_exterior(const orc_cfg* c, const orc_mesh* m, const double* wf, int e,
                         int fp, double* out)
{
    int nv = orc_nv(c), nfp = orc_nfp(c), nf = nfp_face(c);
    int f = fp / nf, k = fp % nf;
    int nb = m->nbr[e * 2 * c->dim + f];
    for (int v = 0; v < nv; v++) {
        if (nb >= 0) out[v] = wf[((size_t)v * m->n_elem + nb) * nfp + (f ^ 1) * nf + k];
        else out[v] = m->bc[(-nb - 1) * nv + v];
    }
}

/* Stencil S of element e (Sec. 5, the "numerical stencil"): its solution
 * points, then its own face points, then the exterior values at the same
 * face points.  S is [|S|][nv]; the first Ns + Nfp rows form the set V. */
void orc_gather_stencil(const orc_cfg* c, const orc_mesh* m, const double* w,
                        const double* wf, int e, double* S)
{
    int nv = orc_nv(c), ns = orc_ns(c), nfp = orc_nfp(c), E = m->n_elem;
    if (c->stencil == 1) {
        /* the wider 1D stencil: own solution points, then those of the left (face 0) and the
         * right (face 1) neighbour; a boundary face contributes its boundary state, once per
         * point (a repeated state changes neither an envelope nor the velocity box) */
        for (int n = 0; n < ns; n++)
            for (int v = 0; v < nv; v++) S[n * nv + v] = w[((size_t)v * E + e) * ns + n];
        for (int f = 0; f < 2; f++) {
            const int nb = m->nbr[e * 2 + f];
            for (int n = 0; n < ns; n++)
                for (int v = 0; v < nv; v++)
                    S[((1 + f) * ns + n) * nv + v] = nb >= 0 ? w[((size_t)v * E + nb) * ns + n]
                                                              : m->bc[(-nb - 1) * nv + v];
        }
        return;
    }
    for (int n = 0; n < ns; n++)
        for (int v = 0; v < nv; v++) S[n * nv + v] = w[((size_t)v * E + e) * ns + n];
    for (int fp = 0; fp < nfp; fp++)
        for (int v = 0; v < nv; v++) S[(ns + fp) * nv + v] = wf[((size_t)v * E + e) * nfp + fp];
    for (int fp = 0; fp < nfp; fp++) orc_exterior(c, m, wf, e, fp, S + (ns + nfp + fp) * nv);
}

int orc_bounds(const orc_cfg* c, const orc_mesh* m, const double* w, const double* wf,
               double* bnd)
{
    int nv = orc_nv(c), nS = orc_nstencil(c), E = m->n_elem;
    double* S = malloc(sizeof(double) * nS * nv);
    int rc = 0;
    for (int e = 0; e < E; e++) {
        double lo[4], hi[4];
        orc_gather_stencil(c, m, w, wf, e, S);
        int r = orc_bounds_stencil(c, nS, S, lo, hi);
        if (r) { rc = r; for (int v = 0; v < nv; v++) { lo[v] = NAN; hi[v] = NAN; } }
        for (int v = 0; v < nv; v++) {
            bnd[(size_t)v * E + e] = lo[v];
            bnd[((size_t)nv + v) * E + e] = hi[v];
        }
    }
    free(S);
    return rc;
}

/* FR right-hand side -div F (Sec. 2.3 and Sec. 5): Gauss-Legendre solution and
 * flux points, the correction functions g_DG, Rusanov common flux, affine
 * Cartesian elements.  Along each axis, at solution point x_i of a line of
 * points:
 *   dF/dxi = sum_m D_im F_m + g_L'(x_i) (Fc_L - F^D_L) + g_R'(x_i) (Fc_R - F^D_R),
 * where F^D is the interpolated discontinuous flux at the face point, and
 * R = -sum_axes (2 / h_axis) dF/dxi. */
void orc_rhs(const orc_cfg* c, const orc_mesh* m, const double* w, const double* wf,
             double* R)
{
    orc_ops o;
    orc_build_ops(c, &o);
    int d = c->dim, nv = o.nv, ns = o.ns, nfp = o.nfp, nf = o.nfpf, n = o.n;
    int E = m->n_elem;
    double* W = malloc(sizeof(double) * ns * nv);
    double* F = malloc(sizeof(double) * d * ns * nv);    /* F[dir][node][v] */
    double* J = malloc(sizeof(double) * nfp * nv);       /* Fc - F^D per face point */
    for (int e = 0; e < E; e++) {
        for (int nd = 0; nd < ns; nd++)
            for (int v = 0; v < nv; v++) W[nd * nv + v] = w[((size_t)v * E + e) * ns + nd];
        for (int dir = 0; dir < d; dir++)
            for (int nd = 0; nd < ns; nd++) orc_flux(c, W + nd * nv, dir, F + (dir * ns + nd) * nv);
        for (int fp = 0; fp < nfp; fp++) {
            int f = fp / nf, k = fp % nf, dir = f / 2, side = f % 2;
            double wi[4], we[4], Fc[4], FD[4];
            for (int v = 0; v < nv; v++) wi[v] = wf[((size_t)v * E + e) * nfp + fp];
            orc_exterior(c, m, wf, e, fp, we);
            if (side == 0) orc_common_flux(c, we, wi, dir, Fc);
            else orc_common_flux(c, wi, we, dir, Fc);
            const double* l = side == 0 ? o.lm : o.lp;
            for (int v = 0; v < nv; v++) {
                double s = 0.0;
                for (int i = 0; i < n; i++) {
                    /* points along this face's normal line through point k */
                    int nd = (d == 1) ? i : (dir == 0 ? k * n + i : i * n + k);
                    s += l[i] * F[(dir * ns + nd) * nv + v];
                }
                FD[v] = s;
                J[fp * nv + v] = Fc[v] - FD[v];
            }
        }
        for (int nd = 0; nd < ns; nd++) {
            int i = (d == 1) ? nd : nd % n, j = (d == 1) ? 0 : nd / n;
            for (int v = 0; v < nv; v++) {
                double dx = 0.0;
                for (int mm = 0; mm < n; mm++) {
                    int q = (d == 1) ? mm : j * n + mm;
                    dx += o.D[i][mm] * F[(0 * ns + q) * nv + v];
                }
                dx += o.gl[i] * J[(0 * nf + j) * nv + v] + o.gr[i] * J[(1 * nf + j) * nv + v];
                double r = -(2.0 / m->h[e * d + 0]) * dx;
                if (d == 2) {
                    double dy = 0.0;
                    for (int mm = 0; mm < n; mm++) dy += o.D[j][mm] * F[(1 * ns + mm * n + i) * nv + v];
                    dy += o.gl[j] * J[(2 * nf + i) * nv + v] + o.gr[j] * J[(3 * nf + i) * nv + v];
                    r -= (2.0 / m->h[e * d + 1]) * dy;
                }
                R[((size_t)v * E + e) * ns + nd] = r;
            }
        }
    }
    free(W); free(F); free(J);
}

/* Limiting of one element's node set, Sec. 3.4 and Sec. 3.8: ns solution values
 * wel[nv][ns] with positive mean weights Wq[ns], nfp face values wfel[nv][nfp].
 *  mean   : positive-quadrature mean sum Wq w / sum Wq (Eq. 13 and assumption
 *           (iii)(a) of Sec. 4)
 *  alpha_i: Eq. 37 per component over V = solution points + face points,
 *           with the epsilon rule stated under it
 *  alpha  : alpha_min = min_i alpha_i (Eq. 39), w~ = mean + alpha (w - mean)
 *           (Eq. 38); at face points w~ = mean + alpha (wf - mean).  With
 *           c->uncoupled each component i takes its own alpha_i instead (the
 *           independent limiting stated after Eq. 39); alpha_out[0] still
 *           reports alpha_min
 *  P      : P_min over V of w~ (Eq. 47); if below p_floor,
 *           alpha_P = |(p_floor - P(mean)) / (P_min - P(mean))| (Eq. 49) and
 *           w~~ = mean + alpha_P (w~ - mean) (Eq. 48).  When P(mean) itself is
 *           not above p_floor, alpha_P is taken as 0. */
void orc_limit_nodes(const orc_cfg* c, int ns, int nfp, const double* Wq, double* wel, const double* wfel,
                     const double* wmin, const double* wmax, double* alpha_out)
{
    int nv = orc_nv(c);
    double mean[4];
    for (int v = 0; v < nv; v++) {
        double s = 0.0, sw = 0.0;
        for (int nd = 0; nd < ns; nd++) {
            s += Wq[nd] * wel[v * ns + nd];
            sw += Wq[nd];
        }
        mean[v] = s / sw;
    }
    double alpha = 1.0, alpha_v[4];
    for (int v = 0; v < nv; v++) {
        double mx = wel[v * ns], mn = wel[v * ns];
        for (int nd = 1; nd < ns; nd++) {
            double x = wel[v * ns + nd];
            if (x > mx) mx = x;
            if (x < mn) mn = x;
        }
        for (int fp = 0; fp < nfp; fp++) {
            double x = wfel[v * nfp + fp];
            if (x > mx) mx = x;
            if (x < mn) mn = x;
        }
        double dmax = mx - mean[v], dmin = mn - mean[v];
        double a;
        if (fabs(dmin) < c->eps || fabs(dmax) < c->eps) {
            a = c->eps_rule ? 1.0 : 0.0;
        } else {
            a = 1.0;
            double t1 = fabs((wmax[v] - mean[v]) / dmax);
            double t2 = fabs((wmin[v] - mean[v]) / dmin);
            if (t1 < a) a = t1;
            if (t2 < a) a = t2;
        }
        alpha_v[v] = a;
        if (a < alpha) alpha = a;
    }
    double* wt = malloc(sizeof(double) * nv * ns);
    double* wtf = malloc(sizeof(double) * nv * nfp);
    for (int v = 0; v < nv; v++) {
        const double av = c->uncoupled ? alpha_v[v] : alpha;
        for (int nd = 0; nd < ns; nd++) wt[v * ns + nd] = mean[v] + av * (wel[v * ns + nd] - mean[v]);
        for (int fp = 0; fp < nfp; fp++) wtf[v * nfp + fp] = mean[v] + av * (wfel[v * nfp + fp] - mean[v]);
    }
    double pmin = INFINITY, q[4];
    for (int nd = 0; nd < ns; nd++) {
        for (int v = 0; v < nv; v++) q[v] = wt[v * ns + nd];
        double P = orc_pressure(c, q);
        if (P < pmin) pmin = P;
    }
    for (int fp = 0; fp < nfp; fp++) {
        for (int v = 0; v < nv; v++) q[v] = wtf[v * nfp + fp];
        double P = orc_pressure(c, q);
        if (P < pmin) pmin = P;
    }
    double aP = 1.0;
    if (pmin < c->p_floor) {
        double Pbar = orc_pressure(c, mean);
        aP = (Pbar > c->p_floor) ? fabs((c->p_floor - Pbar) / (pmin - Pbar)) : 0.0;
        for (int v = 0; v < nv; v++)
            for (int nd = 0; nd < ns; nd++) wel[v * ns + nd] = mean[v] + aP * (wt[v * ns + nd] - mean[v]);
    } else {
        memcpy(wel, wt, sizeof(double) * nv * ns);
    }
    free(wt); free(wtf);
    if (alpha_out) { alpha_out[0] = alpha; alpha_out[1] = aP; }
}

/* The FR element: Gauss-Legendre weights (tensor products in 2D) for the mean. */
void orc_limit_element(const orc_cfg* c, double* wel, const double* wfel,
                       const double* wmin, const double* wmax, double* alpha_out)
{
    int d = c->dim, ns = orc_ns(c), n = c->p + 1;
    double xg[16], wg[16], Wq[256];
    orc_gauss_legendre(n, xg, wg);
    for (int nd = 0; nd < ns; nd++) Wq[nd] = (d == 1) ? wg[nd] : wg[nd % n] * wg[nd / n];
    orc_limit_nodes(c, ns, orc_nfp(c), Wq, wel, wfel, wmin, wmax, alpha_out);
}

void orc_limit(const orc_cfg* c, const orc_mesh* m, double* w, const double* bnd,
               double* alpha)
{
    int nv = orc_nv(c), ns = orc_ns(c), nfp = orc_nfp(c), E = m->n_elem;
    double* wf = malloc(sizeof(double) * (size_t)nv * E * nfp);
    orc_traces(c, m, w, wf);
    double* wel = malloc(sizeof(double) * nv * ns);
    double* wfel = malloc(sizeof(double) * nv * nfp);
    for (int e = 0; e < E; e++) {
        double lo[4], hi[4], a[2];
        for (int v = 0; v < nv; v++) {
            for (int nd = 0; nd < ns; nd++) wel[v * ns + nd] = w[((size_t)v * E + e) * ns + nd];
            for (int fp = 0; fp < nfp; fp++) wfel[v * nfp + fp] = wf[((size_t)v * E + e) * nfp + fp];
            lo[v] = bnd[(size_t)v * E + e];
            hi[v] = bnd[((size_t)nv + v) * E + e];
        }
        orc_limit_element(c, wel, wfel, lo, hi, a);
        for (int v = 0; v < nv; v++)
            for (int nd = 0; nd < ns; nd++) w[((size_t)v * E + e) * ns + nd] = wel[v * ns + nd];
        if (alpha) { alpha[e] = a[0]; alpha[E + e] = a[1]; }
    }
    free(wf); free(wel); free(wfel);
}

/* Shu-Osher form of SSP-RK3 (Gottlieb et al. 2001, as used in Sec. 5):
 *   s = 0: w1 = w_n + dt R(w_n)
 *   s = 1: w2 = 3/4 w_n + 1/4 (w1 + dt R(w1))
 *   s = 2: w3 = 1/3 w_n + 2/3 (w2 + dt R(w2)) */
void orc_stage_combine(const orc_cfg* c, const orc_mesh* m, int s, const double* wn,
                       const double* ws, const double* R, double dt, double* wout)
{
    size_t N = (size_t)orc_nv(c) * m->n_elem * orc_ns(c);
    for (size_t i = 0; i < N; i++) {
        double t = ws[i] + dt * R[i];
        if (s == 0) wout[i] = t;
        else if (s == 1) wout[i] = 0.75 * wn[i] + 0.25 * t;
        else wout[i] = (1.0 / 3.0) * wn[i] + (2.0 / 3.0) * t;
    }
}

/* Time step (the paper does not state its rule): dt = cfl * min over elements,
 * solution points and axes of h_axis / (|U_axis| + c). */
double orc_dt(const orc_cfg* c, const orc_mesh* m, const double* w, double cfl)
{
    int d = c->dim, nv = orc_nv(c), ns = orc_ns(c), E = m->n_elem;
    double best = INFINITY;
    for (int e = 0; e < E; e++) {
        for (int nd = 0; nd < ns; nd++) {
            double q[4];
            for (int v = 0; v < nv; v++) q[v] = w[((size_t)v * E + e) * ns + nd];
            double P = orc_pressure(c, q);
            double a = sqrt(c->gamma * P / q[0]);
            for (int k = 0; k < d; k++) {
                double t = m->h[e * d + k] / (fabs(q[1 + k] / q[0]) + a);
                if (t < best) best = t;
            }
        }
    }
    return cfl * best;
}

/* One time step of the method overview, Sec. 3.9, applied at every SSP-RK3
 * stage: bounds from the stage's input state (steps 1-3), advance (4), limit
 * (5-8). */
int orc_ssprk3_step(const orc_cfg* c, const orc_mesh* m, double* w, double dt,
                    double* alpha)
{
    int nv = orc_nv(c), ns = orc_ns(c), nfp = orc_nfp(c), E = m->n_elem;
    size_t N = (size_t)nv * E * ns;
    double* wn = malloc(sizeof(double) * N);
    double* ws = malloc(sizeof(double) * N);
    double* wo = malloc(sizeof(double) * N);
    double* R = malloc(sizeof(double) * N);
    double* wf = malloc(sizeof(double) * (size_t)nv * E * nfp);
    double* bnd = malloc(sizeof(double) * 2 * (size_t)nv * E);
    memcpy(wn, w, sizeof(double) * N);
    memcpy(ws, w, sizeof(double) * N);
    int rc = 0;
    for (int s = 0; s < 3; s++) {
        orc_traces(c, m, ws, wf);
        int r = orc_bounds(c, m, ws, wf, bnd);
        if (r) rc = r;
        orc_rhs(c, m, ws, wf, R);
        orc_stage_combine(c, m, s, wn, ws, R, dt, wo);
        orc_limit(c, m, wo, bnd, s == 2 ? alpha : NULL);
        memcpy(ws, wo, sizeof(double) * N);
    }
    memcpy(w, ws, sizeof(double) * N);
    free(wn); free(ws); free(wo); free(R); free(wf); free(bnd);
    return rc;
}

/* ===================================================================== */
/* Triangles (Sec. 5: Williams-Shunn solution points, Gauss-Legendre flux */
/* points), affine elements, flux reconstruction with the DG correction.  */
/* ===================================================================== */
/* Reference triangle: vertices (0,0), (1,0), (0,1); (r, s) coordinates; barycentrics
 * (1 - r - s, r, s).  Edge f runs from vertex f to vertex (f + 1) % 3.  Arrays of
 * the triangle path are element-major: w[E][ns][4], wf[E][nfp][4]. */

int orc_tri_ns(int p) { return (p + 1) * (p + 2) / 2; }
int orc_tri_nfp(int p) { return 3 * (p + 1); }

/* Exact integral over the reference triangle of r^i s^j: i! j! / (i + j + 2)!. */
static double orc_tri_monomial_integral(int i, int j)
{
    double num = 1.0, den = 1.0;
    for (int k = 2; k <= i; k++) num *= k;
    for (int k = 2; k <= j; k++) num *= k;
    for (int k = 2; k <= i + j + 2; k++) den *= k;
    return num / den;
}

/* The six points of two symmetric orbits (a, a), (1 - 2a, a), (a, 1 - 2a) with weights W. */
static void orc_tri_orbits6(double a1, double a2, double* rs)
{
    const double a[2] = {a1, a2};
    for (int o = 0; o < 2; o++) {
        rs[(3 * o + 0) * 2 + 0] = a[o];            rs[(3 * o + 0) * 2 + 1] = a[o];
        rs[(3 * o + 1) * 2 + 0] = 1.0 - 2 * a[o];  rs[(3 * o + 1) * 2 + 1] = a[o];
        rs[(3 * o + 2) * 2 + 0] = a[o];            rs[(3 * o + 2) * 2 + 1] = 1.0 - 2 * a[o];
    }
}

/* Residuals of the moment equations of the 6-point rule on r^k, k = 0..4. */
static void orc_tri_res6(const double* x, double* F)
{
    double rs[12];
    orc_tri_orbits6(x[0], x[1], rs);
    for (int k = 0; k < 4; k++) {
        const int deg = k == 0 ? 0 : k + 1;   /* 1, r^2, r^3, r^4 */
        double q = 0.0;
        for (int i = 0; i < 6; i++) q += (i < 3 ? x[2] : x[3]) * pow(rs[2 * i], deg);
        F[k] = q - orc_tri_monomial_integral(deg, 0);
    }
}

/* Williams-Shunn solution points and their quadrature weights on the reference triangle.
 * p = 1: the 3-point interior symmetric rule, barycentric (2/3, 1/6, 1/6), weights 1/6,
 * exact to degree 2.  p = 2: the 6-point rule of two symmetric orbits exact to degree 4 (its
 * four moment equations on 1, r^2, r^3, r^4 fix the two orbit parameters and the two weights),
 * solved by Newton's method with a finite-difference Jacobian from (0.1, 0.45, 0.05, 0.11).
 * rs[ns][2], w[ns]; returns 0, or -2 for another order. */
int orc_tri_points(int p, double* rs, double* w)
{
    if (p == 1) {
        const double a = 1.0 / 6.0;
        rs[0] = a;           rs[1] = a;
        rs[2] = 1.0 - 2 * a; rs[3] = a;
        rs[4] = a;           rs[5] = 1.0 - 2 * a;
        w[0] = w[1] = w[2] = 1.0 / 6.0;
        return 0;
    }
    if (p != 2) return -2;
    double x[4] = {0.1, 0.45, 0.05, 0.11};
    for (int it = 0; it < 60; it++) {
        double F[4], J[4][5];
        orc_tri_res6(x, F);
        double nrm = 0.0;
        for (int k = 0; k < 4; k++) nrm += fabs(F[k]);
        if (nrm < 1e-16) break;
        for (int c = 0; c < 4; c++) {
            double xp[4], Fp[4];
            memcpy(xp, x, sizeof(xp));
            const double hstep = 1e-7 * (fabs(x[c]) + 1e-3);
            xp[c] += hstep;
            orc_tri_res6(xp, Fp);
            for (int k = 0; k < 4; k++) J[k][c] = (Fp[k] - F[k]) / hstep;
        }
        for (int k = 0; k < 4; k++) J[k][4] = -F[k];
        /* Gaussian elimination with partial pivoting */
        for (int c = 0; c < 4; c++) {
            int piv = c;
            for (int r = c + 1; r < 4; r++)
                if (fabs(J[r][c]) > fabs(J[piv][c])) piv = r;
            for (int k = 0; k < 5; k++) { double t = J[c][k]; J[c][k] = J[piv][k]; J[piv][k] = t; }
            for (int r = c + 1; r < 4; r++) {
                const double f = J[r][c] / J[c][c];
                for (int k = c; k < 5; k++) J[r][k] -= f * J[c][k];
            }
        }
        double dx[4];
        for (int c = 3; c >= 0; c--) {
            double t = J[c][4];
            for (int k = c + 1; k < 4; k++) t -= J[c][k] * dx[k];
            dx[c] = t / J[c][c];
        }
        for (int c = 0; c < 4; c++) x[c] += dx[c];
    }
    orc_tri_orbits6(x[0], x[1], rs);
    for (int i = 0; i < 6; i++) w[i] = i < 3 ? x[2] : x[3];
    return 0;
}

/* Monomials r^a s^b with a + b <= p, in the order a + b = 0, 1, ..., p and a descending. */
static int orc_tri_monomials(int p, int* ea, int* eb)
{
    int n = 0;
    for (int d = 0; d <= p; d++)
        for (int a = d; a >= 0; a--) { ea[n] = a; eb[n] = d - a; n++; }
    return n;
}

typedef struct {
    int p, ns, nfp;
    double rs[6][2], wq[6];          /* solution points, weights (sum 1/2) */
    double C[6][6];                  /* phi_j = sum_m C[m][j] r^a_m s^b_m */
    double fr[9][2];                 /* flux points (reference) */
    double gw[9];                    /* Gauss-Legendre weight of each flux point (sum 2 per edge) */
    double phi_f[9][6];              /* phi_j at the flux points */
    double dr[6][6], ds[6][6];       /* d phi_j / dr, / ds at the solution points [i][j] */
} orc_triops;

static double orc_tri_phi(const orc_triops* o, int j, double r, double s, int dr, int ds)
{
    int ea[6], eb[6];
    const int n = orc_tri_monomials(o->p, ea, eb);
    double v = 0.0;
    for (int m = 0; m < n; m++) {
        int a = ea[m], b = eb[m];
        double coef = o->C[m][j];
        if (dr) { if (a == 0) continue; coef *= a; a -= 1; }
        if (ds) { if (b == 0) continue; coef *= b; b -= 1; }
        v += coef * pow(r, a) * pow(s, b);
    }
    return v;
}

/* The Lagrange basis of the solution points (inverse of the monomial Vandermonde matrix by
 * Gauss-Jordan elimination), its derivatives at the solution points, its values at the flux
 * points (p + 1 Gauss-Legendre points on each edge, in the edge's direction). */
static int orc_tri_build_ops(int p, orc_triops* o)
{
    if (p < 1 || p > 2) return -2;
    o->p = p;
    o->ns = orc_tri_ns(p);
    o->nfp = orc_tri_nfp(p);
    double rs[12], wq[6];
    orc_tri_points(p, rs, wq);
    int ea[6], eb[6];
    const int n = orc_tri_monomials(p, ea, eb);
    double A[6][12];
    for (int i = 0; i < n; i++) {
        o->rs[i][0] = rs[2 * i];
        o->rs[i][1] = rs[2 * i + 1];
        o->wq[i] = wq[i];
        for (int m = 0; m < n; m++) A[i][m] = pow(rs[2 * i], ea[m]) * pow(rs[2 * i + 1], eb[m]);
        for (int m = 0; m < n; m++) A[i][n + m] = (i == m) ? 1.0 : 0.0;
    }
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int k = 0; k < 2 * n; k++) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        const double d = A[c][c];
        for (int k = 0; k < 2 * n; k++) A[c][k] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            const double f = A[r][c];
            for (int k = 0; k < 2 * n; k++) A[r][k] -= f * A[c][k];
        }
    }
    /* V C = I with V[i][m] = mono_m(x_i): C = V^-1 is the right half */
    for (int m = 0; m < n; m++)
        for (int j = 0; j < n; j++) o->C[m][j] = A[m][n + j];
    double xg[8], wg[8];
    orc_gauss_legendre(p + 1, xg, wg);
    const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    for (int f = 0; f < 3; f++)
        for (int k = 0; k <= p; k++) {
            const double t = 0.5 * (1.0 + xg[k]);
            const int q = f * (p + 1) + k;
            o->fr[q][0] = V[f][0] + t * (V[(f + 1) % 3][0] - V[f][0]);
            o->fr[q][1] = V[f][1] + t * (V[(f + 1) % 3][1] - V[f][1]);
            o->gw[q] = wg[k];
        }
    for (int q = 0; q < o->nfp; q++)
        for (int j = 0; j < n; j++) o->phi_f[q][j] = orc_tri_phi(o, j, o->fr[q][0], o->fr[q][1], 0, 0);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            o->dr[i][j] = orc_tri_phi(o, j, o->rs[i][0], o->rs[i][1], 1, 0);
            o->ds[i][j] = orc_tri_phi(o, j, o->rs[i][0], o->rs[i][1], 0, 1);
        }
    return 0;
}

/* Affine geometry of element e: x = X0 + J (r, s), J = [X1 - X0 | X2 - X0]; the inverse
 * Jacobian rows (dr/dx, dr/dy), (ds/dx, ds/dy); det J; edge lengths; outward unit normals
 * (the vertices run counterclockwise: the outward normal of edge (dx, dy) is (dy, -dx) / L). */
typedef struct { double rx, ry, sx, sy, det, len[3], nx[3], ny[3]; } orc_trigeo;

static void orc_tri_geometry(const orc_trimesh* m, int e, orc_trigeo* g)
{
    const double* X = m->xy + (size_t)e * 6;
    const double J00 = X[2] - X[0], J10 = X[3] - X[1], J01 = X[4] - X[0], J11 = X[5] - X[1];
    g->det = J00 * J11 - J01 * J10;
    g->rx = J11 / g->det;  g->ry = -J01 / g->det;
    g->sx = -J10 / g->det; g->sy = J00 / g->det;
    for (int f = 0; f < 3; f++) {
        const double dx = X[2 * ((f + 1) % 3)] - X[2 * f], dy = X[2 * ((f + 1) % 3) + 1] - X[2 * f + 1];
        g->len[f] = sqrt(dx * dx + dy * dy);
        g->nx[f] = dy / g->len[f];
        g->ny[f] = -dx / g->len[f];
    }
}

/* Curved elements: x(r, s) = sum_k N_k(r, s) X_k with the six quadratic Lagrange shape
 * functions of the corners and the edge mid-parameter points (barycentrics l1 = 1 - r - s,
 * l2 = r, l3 = s: N0 = l1 (2 l1 - 1), N1 = l2 (2 l2 - 1), N2 = l3 (2 l3 - 1), N3 = 4 l1 l2,
 * N4 = 4 l2 l3, N5 = 4 l3 l1); the derivatives x_r, x_s, y_r, y_s of the map at (r, s). */
static void orc_tri_map_deriv(const double* X, double r, double s, double* xr, double* xs, double* yr, double* ys)
{
    const double l1 = 1.0 - r - s, l2 = r, l3 = s;
    const double dr[6] = {-(4.0 * l1 - 1.0), 4.0 * l2 - 1.0, 0.0, 4.0 * (l1 - l2), 4.0 * l3, -4.0 * l3};
    const double ds[6] = {-(4.0 * l1 - 1.0), 0.0, 4.0 * l3 - 1.0, -4.0 * l2, 4.0 * l2, 4.0 * (l1 - l3)};
    *xr = *xs = *yr = *ys = 0.0;
    for (int k = 0; k < 6; k++) {
        *xr += dr[k] * X[2 * k];
        *xs += ds[k] * X[2 * k];
        *yr += dr[k] * X[2 * k + 1];
        *ys += ds[k] * X[2 * k + 1];
    }
}

/* Interior values at the flux points: interpolation of the solution polynomial. */
void orc_tri_traces(const orc_cfg* c, const orc_trimesh* m, const double* w, double* wf)
{
    orc_triops o;
    if (orc_tri_build_ops(c->p, &o)) return;
    for (int e = 0; e < m->n_elem; e++)
        for (int q = 0; q < o.nfp; q++)
            for (int v = 0; v < 4; v++) {
                double s = 0.0;
                for (int j = 0; j < o.ns; j++) s += o.phi_f[q][j] * w[((size_t)e * o.ns + j) * 4 + v];
                wf[((size_t)e * o.nfp + q) * 4 + v] = s;
            }
}

/* Exterior value at flux point k of edge f of element e: the neighbour's interior value at the
 * same point (its matched edge runs the other way: its point p - k), or the boundary state. */
static void orc_tri_exterior(const orc_trimesh* m, int p, const double* wf, int e, int f, int k, double* q)
{
    const int nb = m->nbr[e * 3 + f];
    if (nb >= 0) {
        const int g = m->nbr_edge[e * 3 + f];
        const double* src = wf + ((size_t)nb * 3 * (p + 1) + g * (p + 1) + (p - k)) * 4;
        for (int v = 0; v < 4; v++) q[v] = src[v];
    } else {
        for (int v = 0; v < 4; v++) q[v] = m->bc[(-nb - 1) * 4 + v];
    }
}

/* The stencil of Sec. 5 for a triangle: its solution points, its flux points, the exterior
 * values at the flux points; S[ns + 2 nfp][4]. */
void orc_tri_gather_stencil(const orc_cfg* c, const orc_trimesh* m, const double* w, const double* wf, int e,
                            double* S)
{
    const int p = c->p, ns = orc_tri_ns(p), nfp = orc_tri_nfp(p);
    for (int i = 0; i < ns; i++)
        for (int v = 0; v < 4; v++) S[i * 4 + v] = w[((size_t)e * ns + i) * 4 + v];
    for (int q = 0; q < nfp; q++)
        for (int v = 0; v < 4; v++) S[(ns + q) * 4 + v] = wf[((size_t)e * nfp + q) * 4 + v];
    for (int f = 0; f < 3; f++)
        for (int k = 0; k <= p; k++) orc_tri_exterior(m, p, wf, e, f, k, S + (ns + nfp + f * (p + 1) + k) * 4);
}

/* Common flux along the outward normal n of an edge, qi inside, qe outside: the configured 1D
 * flux (Rusanov, HLLC or HLL) of the states rotated into the (n, t) frame, t = (-n_y, n_x),
 * with the interior state on the minus side, and its momentum part rotated back. */
static void orc_tri_common_flux(const orc_cfg* c, const double* qi, const double* qe, double nx, double ny,
                                double* F)
{
    const double li[4] = {qi[0], qi[1] * nx + qi[2] * ny, -qi[1] * ny + qi[2] * nx, qi[3]};
    const double le[4] = {qe[0], qe[1] * nx + qe[2] * ny, -qe[1] * ny + qe[2] * nx, qe[3]};
    double Fl[4];
    orc_common_flux(c, li, le, 0, Fl);
    F[0] = Fl[0];
    F[1] = Fl[1] * nx - Fl[2] * ny;
    F[2] = Fl[1] * ny + Fl[2] * nx;
    F[3] = Fl[3];
}

/* The residual of a curved element (FR with the DG correction on the mapped element, the
 * transformed-flux form): with adj J = |J| J^-1 at each point, the transformed flux
 * Ft = adj J F, and at each flux point the reference unit normal nh of its edge, the physical
 * unit normal n and the stretch sigma = |dx/dt| / |dxi/dt| along the edge (Nanson: Ft . nh =
 * sigma F . n),
 *   R_i = -(1/|J_i|) [ sum_j (Dr_ij Ft_r,j + Ds_ij Ft_s,j)
 *                      + sum_q phi_i(x_q) gw_q L_f / (2 w_i) (sigma_q F*_n,q - (Ft_h . nh)(x_q)) ],
 * L_f the reference edge's length.  The solution points carry the lumped mass w_i |J_i| (the
 * collocated quadrature of FR; exact for affine elements). */
static void orc_tri_rhs_curved(const orc_cfg* c, const orc_trimesh* m, const orc_triops* o, int e,
                               double Fx[6][4], double Fy[6][4], const double* wf, double* Re)
{
    const int ns = o->ns, nfp = o->nfp, p = c->p;
    const double* X = m->xy6 + (size_t)e * 12;
    double Fr[6][4], Fs[6][4], detJ[6];
    for (int j = 0; j < ns; j++) {
        double xr, xs, yr, ys;
        orc_tri_map_deriv(X, o->rs[j][0], o->rs[j][1], &xr, &xs, &yr, &ys);
        detJ[j] = xr * ys - xs * yr;
        for (int v = 0; v < 4; v++) {
            Fr[j][v] = ys * Fx[j][v] - xs * Fy[j][v];
            Fs[j][v] = -yr * Fx[j][v] + xr * Fy[j][v];
        }
    }
    double acc[6][4];
    for (int i = 0; i < ns; i++)
        for (int v = 0; v < 4; v++) {
            double d = 0.0;
            for (int j = 0; j < ns; j++) d += o->dr[i][j] * Fr[j][v] + o->ds[i][j] * Fs[j][v];
            acc[i][v] = d;
        }
    const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    for (int f = 0; f < 3; f++) {
        const double dvx = V[(f + 1) % 3][0] - V[f][0], dvy = V[(f + 1) % 3][1] - V[f][1];
        const double L = sqrt(dvx * dvx + dvy * dvy);
        const double nhx = dvy / L, nhy = -dvx / L;
        for (int k = 0; k <= p; k++) {
            const int q = f * (p + 1) + k;
            double xr, xs, yr, ys;
            orc_tri_map_deriv(X, o->fr[q][0], o->fr[q][1], &xr, &xs, &yr, &ys);
            const double tx = xr * dvx + xs * dvy, ty = yr * dvx + ys * dvy;
            const double ds = sqrt(tx * tx + ty * ty);
            const double nx = ty / ds, ny = -tx / ds, sigma = ds / L;
            double qe[4], Fstar[4];
            orc_tri_exterior(m, p, wf, e, f, k, qe);
            orc_tri_common_flux(c, wf + ((size_t)e * nfp + q) * 4, qe, nx, ny, Fstar);
            for (int v = 0; v < 4; v++) {
                double Fn = 0.0;
                for (int j = 0; j < ns; j++) Fn += o->phi_f[q][j] * (Fr[j][v] * nhx + Fs[j][v] * nhy);
                const double jump = sigma * Fstar[v] - Fn;
                for (int i = 0; i < ns; i++) acc[i][v] += o->phi_f[q][i] * o->gw[q] * L / (2.0 * o->wq[i]) * jump;
            }
        }
    }
    for (int i = 0; i < ns; i++)
        for (int v = 0; v < 4; v++) Re[i * 4 + v] = -acc[i][v] / detJ[i];
}

/* Mean weights of element e for the limiter: the lumped mass w_i |J_i| of a curved element, the
 * rule's weights w_i of an affine one (the same mean: |J| is constant there). */
static void orc_tri_mean_weights(const orc_trimesh* m, const orc_triops* o, int e, double* W)
{
    for (int i = 0; i < o->ns; i++) {
        W[i] = o->wq[i];
        if (m->xy6) {
            double xr, xs, yr, ys;
            orc_tri_map_deriv(m->xy6 + (size_t)e * 12, o->rs[i][0], o->rs[i][1], &xr, &xs, &yr, &ys);
            W[i] *= xr * ys - xs * yr;
        }
    }
}

/* Strong-form nodal DG residual (FR with the DG correction) of an affine triangle:
 *   R_i = -div F_h(x_i) - sum_q phi_i(x_q) (|e_q| gw_q / 2) / (det J w_i) (F*_n - F_h . n)(x_q)
 * with F_h the interpolation of the solution-point fluxes (Eq. 2), x_q the flux points and
 * F*_n the common normal flux.  The Williams-Shunn rule integrates the degree-2p products
 * phi_i phi_j exactly, so the mass matrix is diag(det J w_i) and the lifting above is exact. */
void orc_tri_rhs(const orc_cfg* c, const orc_trimesh* m, const double* w, const double* wf, double* R)
{
    orc_triops o;
    if (orc_tri_build_ops(c->p, &o)) return;
    const int ns = o.ns, nfp = o.nfp, p = c->p;
    for (int e = 0; e < m->n_elem; e++) {
        orc_trigeo g;
        orc_tri_geometry(m, e, &g);
        double Fx[6][4], Fy[6][4];
        for (int j = 0; j < ns; j++) {
            orc_flux(c, w + ((size_t)e * ns + j) * 4, 0, Fx[j]);
            orc_flux(c, w + ((size_t)e * ns + j) * 4, 1, Fy[j]);
        }
        if (m->xy6) {
            orc_tri_rhs_curved(c, m, &o, e, Fx, Fy, wf, R + (size_t)e * ns * 4);
            continue;
        }
        for (int i = 0; i < ns; i++)
            for (int v = 0; v < 4; v++) {
                double div = 0.0;
                for (int j = 0; j < ns; j++) {
                    const double dx = o.dr[i][j] * g.rx + o.ds[i][j] * g.sx;
                    const double dy = o.dr[i][j] * g.ry + o.ds[i][j] * g.sy;
                    div += dx * Fx[j][v] + dy * Fy[j][v];
                }
                R[((size_t)e * ns + i) * 4 + v] = -div;
            }
        for (int f = 0; f < 3; f++)
            for (int k = 0; k <= p; k++) {
                const int q = f * (p + 1) + k;
                double qe[4], Fs[4];
                orc_tri_exterior(m, p, wf, e, f, k, qe);
                orc_tri_common_flux(c, wf + ((size_t)e * nfp + q) * 4, qe, g.nx[f], g.ny[f], Fs);
                for (int v = 0; v < 4; v++) {
                    double Fn = 0.0;
                    for (int j = 0; j < ns; j++) Fn += o.phi_f[q][j] * (Fx[j][v] * g.nx[f] + Fy[j][v] * g.ny[f]);
                    const double jump = Fs[v] - Fn;
                    for (int i = 0; i < ns; i++)
                        R[((size_t)e * ns + i) * 4 + v] -= o.phi_f[q][i] * (0.5 * g.len[f] * o.gw[q]) /
                                                           (g.det * o.wq[i]) * jump;
                }
            }
    }
}

/* Time step on triangles (the paper states no rule): cfl * min over elements and solution
 * points of h_e / (|U| + c), h_e = 2 area / longest edge (the shortest altitude). */
double orc_tri_dt(const orc_cfg* c, const orc_trimesh* m, const double* w, double cfl)
{
    const int ns = orc_tri_ns(c->p);
    double best = INFINITY;
    for (int e = 0; e < m->n_elem; e++) {
        orc_trigeo g;
        orc_tri_geometry(m, e, &g);
        double lmax = g.len[0];
        if (g.len[1] > lmax) lmax = g.len[1];
        if (g.len[2] > lmax) lmax = g.len[2];
        const double h = g.det / lmax;   /* 2 (det / 2) / longest edge */
        for (int i = 0; i < ns; i++) {
            const double* q = w + ((size_t)e * ns + i) * 4;
            const double P = orc_pressure(c, q);
            const double u = sqrt(q[1] * q[1] + q[2] * q[2]) / q[0];
            const double t = h / (u + sqrt(c->gamma * P / q[0]));
            if (t < best) best = t;
        }
    }
    return cfl * best;
}

/* One SSP-RK3 step on triangles, limited after every stage as on quads (Sec. 3.9, Sec. 5):
 * bounds of each element's stencil (orc_bounds_stencil), the residual, the Shu-Osher
 * combination, then the limiter of the node set (orc_limit_nodes) with the element's mean
 * weights (the Williams-Shunn weights, times |J_i| on a curved element) and the flux-point
 * values of the combined state. */
int orc_tri_ssprk3_step(const orc_cfg* c, const orc_trimesh* m, double* w, double dt, double* alpha)
{
    const int p = c->p, ns = orc_tri_ns(p), nfp = orc_tri_nfp(p), E = m->n_elem, nst = ns + 2 * nfp;
    if (p < 1 || p > 2) return -2;
    orc_triops o;
    orc_tri_build_ops(p, &o);
    const size_t N = (size_t)E * ns * 4;
    double* wn = malloc(sizeof(double) * N);
    double* ws = malloc(sizeof(double) * N);
    double* R = malloc(sizeof(double) * N);
    double* wf = malloc(sizeof(double) * (size_t)E * nfp * 4);
    double* lo = malloc(sizeof(double) * (size_t)E * 4);
    double* hi = malloc(sizeof(double) * (size_t)E * 4);
    double S[64 * 4], wel[4 * 6], wfel[4 * 9];
    memcpy(wn, w, sizeof(double) * N);
    memcpy(ws, w, sizeof(double) * N);
    int rc = 0;
    for (int s = 0; s < 3; s++) {
        orc_tri_traces(c, m, ws, wf);
        for (int e = 0; e < E; e++) {
            orc_tri_gather_stencil(c, m, ws, wf, e, S);
            const int r = orc_bounds_stencil(c, nst, S, lo + 4 * e, hi + 4 * e);
            if (r) rc = r;
        }
        orc_tri_rhs(c, m, ws, wf, R);
        for (size_t i = 0; i < N; i++) {
            const double t = ws[i] + dt * R[i];
            ws[i] = s == 0 ? t : (s == 1 ? 0.75 * wn[i] + 0.25 * t : (1.0 / 3.0) * wn[i] + (2.0 / 3.0) * t);
        }
        orc_tri_traces(c, m, ws, wf);
        for (int e = 0; e < E; e++) {
            double a[2];
            for (int v = 0; v < 4; v++) {
                for (int i = 0; i < ns; i++) wel[v * ns + i] = ws[((size_t)e * ns + i) * 4 + v];
                for (int q = 0; q < nfp; q++) wfel[v * nfp + q] = wf[((size_t)e * nfp + q) * 4 + v];
            }
            double W[6];
            orc_tri_mean_weights(m, &o, e, W);
            orc_limit_nodes(c, ns, nfp, W, wel, wfel, lo + 4 * e, hi + 4 * e, a);
            for (int v = 0; v < 4; v++)
                for (int i = 0; i < ns; i++) ws[((size_t)e * ns + i) * 4 + v] = wel[v * ns + i];
            if (alpha && s == 2) { alpha[e] = a[0]; alpha[E + e] = a[1]; }
        }
    }
    memcpy(w, ws, sizeof(double) * N);
    free(wn); free(ws); free(R); free(wf); free(lo); free(hi);
    return rc;
}
