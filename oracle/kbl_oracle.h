/*
 * kbl_oracle.h -- plain, slow, FP64 CPU restatement of the kinetic-bounds
 * limiter of Dzanic & Martinelli, "High-order limiting methods using maximum
 * principle bounds derived from the Boltzmann equation I: Euler equations"
 * (arXiv 2407.20966), together with the nodal DG / flux-reconstruction Euler
 * stage around it.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  It
 * shares no source, header, table or helper with the CUDA path; only tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Conventions (shared by the whole file):
 *   d      spatial dimension (1 or 2), nv = d + 2 conserved components
 *          ordered (rho, m_x[, m_y], E).
 *   p      polynomial order; Gauss-Legendre solution points, (p+1)^d per
 *          element, x index fastest: node n = j*(p+1) + i.
 *   faces  1D: 0 = -x, 1 = +x (one point each).  2D: 0 = -x, 1 = +x, 2 = -y,
 *          3 = +y, each with p+1 Gauss-Legendre points ordered by increasing
 *          coordinate along the face.  Face point f*nfpf + k.
 *   arrays solution  w [nv][E][Ns]      (SoA, element-major inside a variable)
 *          traces    wf[nv][E][Nfp]     (interior value at each face point)
 *          bounds    bnd[2][nv][E]      (bnd[0] = minimum, bnd[1] = maximum)
 *   mesh   axis-aligned Cartesian elements.  nbr[E][2d] >= 0 is the element on
 *          the other side of face f (matched to its face f^1, same point
 *          order); nbr < 0 marks a boundary face whose exterior state is the
 *          prescribed conserved state bc[-(nbr+1)][nv].
 *
 * Return codes: 0 success, -1 a non-physical state (rho <= 0 or P <= 0) was
 * met, -2 bad argument.
 */
#ifndef KBL_ORACLE_H
#define KBL_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;          /* d */
    int p;            /* polynomial order */
    int nu[2];        /* velocity points per dimension (nu[1] unused in 1D) */
    double gamma;     /* ratio of specific heats */
    double k;         /* half-width of the velocity box in thermal units, Eq. 45 */
    double r_fac;     /* relaxation factor, Eq. 40 (0 = strict bounds) */
    double eps;       /* threshold of the alpha rule under Eq. 37 */
    double rho_floor; /* density floor, Sec. 3.8 */
    double p_floor;   /* pressure floor, Sec. 3.8 */
    int eps_rule;     /* 0: alpha_i = 0 when |extremum - mean| < eps (as printed);
                         1: the component is skipped (alpha_i = 1) */
    int uncoupled;    /* 0: every component takes alpha_min = min_i alpha_i (Eq. 38-39, the
                         paper's choice); 1: each component its own alpha_i (the independent
                         option stated after Eq. 39) */
    int flux;         /* common flux: 0 Rusanov (the flux of the analysis, Sec. 4), 1 HLLC
                         (the flux of the experiments, Sec. 5), 2 HLL (the Sedov run, Sec. 6.6) */
    int quadrature;   /* velocity quadrature: 0 trapezoidal (Sec. 3.7), 1 Romberg (named in
                         Sec. 5; needs nu - 1 even on every axis) */
    int stencil;      /* 0: the numerical stencil of Sec. 5 (own solution and face points, the
                         exterior face values); 1 (1D only): the element's own solution points
                         and all solution points of both face neighbours */
} orc_cfg;

typedef struct {
    int n_elem;
    const int* nbr;    /* [E][2d] */
    const double* h;   /* [E][d] element widths */
    int n_bc;
    const double* bc;  /* [n_bc][nv] */
} orc_mesh;

/* ---- counts ---------------------------------------------------------- */
int orc_nv(const orc_cfg* c);
int orc_ns(const orc_cfg* c);        /* solution points per element */
int orc_nfp(const orc_cfg* c);       /* face points per element */
int orc_nstencil(const orc_cfg* c);  /* |S| = Ns + 2 Nfp (stencil 0), 3 Ns (stencil 1) */

/* ---- one-dimensional polynomial tools (Sec. 2.3, Sec. 5) ------------- */
void orc_legendre(int n, double x, double* P, double* dP);
int orc_gauss_legendre(int n, double* x, double* w);
double orc_lagrange(int n, const double* nodes, int j, double x);
double orc_lagrange_deriv(int n, const double* nodes, int j, double x);
void orc_correction_deriv(int p, double x, double* dgl, double* dgr);

/* ---- Euler physics (Eq. 2, Eq. 3) ------------------------------------ */
double orc_pressure(const orc_cfg* c, const double* w);
void orc_flux(const orc_cfg* c, const double* w, int dir, double* F);
void orc_hllc(const orc_cfg* c, const double* wl, const double* wr, int dir, double* F);
void orc_hll(const orc_cfg* c, const double* wl, const double* wr, int dir, double* F);
double orc_romberg_weight(int N, int j);
void orc_rusanov(const orc_cfg* c, const double* wl, const double* wr, int dir,
                 double* F);

/* ---- kinetic bounds (Sec. 3.3 - 3.8) ---------------------------------- */
/* Bounds over one stencil S given as S[nS][nv].  wmin/wmax get nv values. */
int orc_bounds_stencil(const orc_cfg* c, int nS, const double* S, double* wmin,
                       double* wmax);
/* Quadrature moments of the Maxwellian of stencil state `which`, on the same
 * velocity grid and with the same summation order orc_bounds_stencil uses
 * for S. */
int orc_state_moments(const orc_cfg* c, int nS, const double* S, int which,
                      double* mom);
/* Plain moments (rho, m, E) of the relaxed envelope f_min (upper = 0) or
 * f_max (upper = 1) of S, taken as distributions in their own right. */
int orc_envelope_moments(const orc_cfg* c, int nS, const double* S, int upper,
                         double* mom);
/* Velocity box of S (Eq. 45): lo[d], hi[d]. */
int orc_velocity_box(const orc_cfg* c, int nS, const double* S, double* lo,
                     double* hi);

/* ---- mesh-level operations ------------------------------------------- */
void orc_traces(const orc_cfg* c, const orc_mesh* m, const double* w, double* wf);
void orc_gather_stencil(const orc_cfg* c, const orc_mesh* m, const double* w,
                        const double* wf, int e, double* S);
int orc_bounds(const orc_cfg* c, const orc_mesh* m, const double* w,
               const double* wf, double* bnd);
void orc_rhs(const orc_cfg* c, const orc_mesh* m, const double* w,
             const double* wf, double* R);
/* Limit one element: wel[nv][Ns] in place; wfel[nv][Nfp] are its unlimited
 * face values.  alpha_out[0] = alpha_min (Eq. 39), alpha_out[1] = alpha_P
 * (Eq. 49, 1 when the pressure step is not taken). */
void orc_limit_nodes(const orc_cfg* c, int ns, int nfp, const double* Wq, double* wel, const double* wfel,
                     const double* wmin, const double* wmax, double* alpha_out);
void orc_limit_element(const orc_cfg* c, double* wel, const double* wfel,
                       const double* wmin, const double* wmax, double* alpha_out);
void orc_limit(const orc_cfg* c, const orc_mesh* m, double* w, const double* bnd,
               double* alpha /* [2][E] or NULL */);
/* SSP-RK3 stage combination (Shu-Osher form), stage s in {0,1,2}. */
void orc_stage_combine(const orc_cfg* c, const orc_mesh* m, int s, const double* wn,
                       const double* ws, const double* R, double dt, double* wout);
double orc_dt(const orc_cfg* c, const orc_mesh* m, const double* w, double cfl);
/* One SSP-RK3 step with bounds and limiting after every stage (Sec. 3.9). */
int orc_ssprk3_step(const orc_cfg* c, const orc_mesh* m, double* w, double dt,
                    double* alpha /* [2][E] of the last stage, or NULL */);

/* ---- triangles (Sec. 5), affine elements, element-major arrays ------- */
typedef struct {
    int n_elem;
    const double* xy;     /* [E][3][2] vertices, counterclockwise */
    const int* nbr;       /* [E][3] element across edge f (vertex f to (f+1)%3), < 0 boundary id -(nbr+1) */
    const int* nbr_edge;  /* [E][3] the neighbour's edge matched to edge f */
    int n_bc;
    const double* bc;     /* [n_bc][4] */
    const double* xy6;    /* curved (quadratic) elements, or NULL for affine ones: [E][6][2], the
                             corners (as in xy) then the points of edges 0, 1, 2 at mid-parameter */
} orc_trimesh;

int orc_tri_ns(int p);    /* (p+1)(p+2)/2 solution points */
int orc_tri_nfp(int p);   /* 3 (p+1) flux points */
int orc_tri_points(int p, double* rs, double* w);
void orc_tri_traces(const orc_cfg* c, const orc_trimesh* m, const double* w, double* wf);
void orc_tri_gather_stencil(const orc_cfg* c, const orc_trimesh* m, const double* w, const double* wf, int e,
                            double* S);
void orc_tri_rhs(const orc_cfg* c, const orc_trimesh* m, const double* w, const double* wf, double* R);
double orc_tri_dt(const orc_cfg* c, const orc_trimesh* m, const double* w, double cfl);
int orc_tri_ssprk3_step(const orc_cfg* c, const orc_trimesh* m, double* w, double dt, double* alpha);

#ifdef __cplusplus
}
#endif
#endif
