// kbl_tri.cu -- the method on affine triangles (Sec. 5: Williams-Shunn solution points,
// Gauss-Legendre flux points), FP64 flux reconstruction with the DG correction, and the SSP-RK3
// step that feeds the element-agnostic bounds (kbl_bounds_stencil) and node-set limiter
// (kbl_limit_nodes).
//
// Reference triangle (0,0), (1,0), (0,1); barycentrics (l1, l2, l3) = (1 - r - s, r, s).  Edge f
// runs from vertex f to vertex (f + 1) % 3 with p + 1 Gauss-Legendre flux points in its
// direction; the element across it runs the shared edge the other way (its point p - k).
// Arrays are element-major: w[E][ns][4], traces wf[E][nfp][4], stencils S[E][ns + 2 nfp][4].
//
// Solution points: the Williams-Shunn points of orders 1 and 2 are the unique interior
// symmetric rules of 3 points (degree 2) and 6 points in two orbits (degree 4).  They are found
// here from their symmetric moment equations (the invariants 1, e2, e3, e2^2 of the
// barycentrics) by Newton's method with an analytic Jacobian.  The rule integrates the degree-2p
// products of the Lagrange basis exactly, so the nodal mass matrix is diag(det J w_i) and the
// lifting of the DG correction at flux point q is phi_i(x_q) (|e_q| gw_q / 2) / (det J w_i).
//
// Residual (Sec. 2.3 on simplices): R_i = -div F_h(x_i) - sum_q lift_iq (F*_n - F_h . n)(x_q),
// F_h the interpolation of the solution-point fluxes, F*_n the configured common flux of the
// states rotated into the edge's (n, t) frame.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kbl_fr_body.cuh"

namespace {

constexpr int TRI_PMAX = 2, TRI_NSMAX = 6, TRI_NFPMAX = 9;

struct TriOps {
    int p, ns, nfp;
    double wq[TRI_NSMAX];                 // rule weights (sum 1/2)
    double dr[TRI_NSMAX][TRI_NSMAX];      // d phi_j / dr at solution point i: [i][j]
    double ds[TRI_NSMAX][TRI_NSMAX];
    double phif[TRI_NFPMAX][TRI_NSMAX];   // phi_j at flux point q
    double gw[TRI_NFPMAX];                // Gauss-Legendre weight of flux point q (sum 2 per edge)
    double lift[TRI_NFPMAX][TRI_NSMAX];   // phi_i(x_q) gw_q / (2 w_i): the lifting without |e| / det J
    // FP32 copies (rounded on the host) for the FP32 arithmetic of the mixed precision
    float drf[TRI_NSMAX][TRI_NSMAX], dsf[TRI_NSMAX][TRI_NSMAX], phiff[TRI_NFPMAX][TRI_NSMAX],
        liftf[TRI_NFPMAX][TRI_NSMAX];
};

// Per element: inverse Jacobian (dr/dx, dr/dy, ds/dx, ds/dy), det J, edge lengths, outward
// unit normals, h = det J / longest edge (the shortest altitude).
struct TriGeo {
    double rx, ry, sx, sy, det, len[3], nx[3], ny[3], h;
};

// ---- host: the rule and the basis ------------------------------------------
// Symmetric-orbit points (a, a), (1 - 2a, a), (a, 1 - 2a) in (r, s); their barycentrics are the
// permutations of (1 - 2a, a, a).  Invariant moments of one orbit (sum over its 3 points) of
// e2 = l1 l2 + l1 l3 + l2 l3, e3 = l1 l2 l3, e2^2 and their a-derivatives.
void orbit_moments(double a, double m[4], double dm[4])
{
    const double b = 1.0 - 2.0 * a, db = -2.0;
    const double e2 = 2.0 * a * b + a * a, de2 = 2.0 * (b + a * db) + 2.0 * a;
    const double e3 = a * a * b, de3 = 2.0 * a * b + a * a * db;
    m[0] = 3.0;
    m[1] = 3.0 * e2;
    m[2] = 3.0 * e3;
    m[3] = 3.0 * e2 * e2;
    dm[0] = 0.0;
    dm[1] = 3.0 * de2;
    dm[2] = 3.0 * de3;
    dm[3] = 6.0 * e2 * de2;
}

// Exact integrals over the reference triangle of 1, e2, e3, e2^2 (sums of
// int l1^i l2^j l3^k = i! j! k! / (i + j + k + 2)!).
void invariant_integrals(double I[4])
{
    I[0] = 0.5;
    I[1] = 3.0 * (1.0 / 24.0);                       // 3 x int l1 l2
    I[2] = 1.0 / 120.0;                              // int l1 l2 l3
    // e2^2 = sum l_i^2 l_j^2 (3 terms) + 2 sum over pairs of products sharing a factor:
    //   2 (l1^2 l2 l3 + l1 l2^2 l3 + l1 l2 l3^2)
    I[3] = 3.0 * (2.0 * 2.0 / 720.0) + 2.0 * 3.0 * (2.0 / 720.0);
}

bool ws_points(int p, double rs[][2], double* w)
{
    if (p == 1) {
        const double a = 1.0 / 6.0;   // the interior 3-point rule of degree 2 (one orbit, equal weights)
        const double pts[3][2] = {{a, a}, {1.0 - 2.0 * a, a}, {a, 1.0 - 2.0 * a}};
        for (int i = 0; i < 3; i++) {
            rs[i][0] = pts[i][0];
            rs[i][1] = pts[i][1];
            w[i] = 1.0 / 6.0;
        }
        return true;
    }
    if (p != 2) return false;
    // unknowns x = (a1, a2, W1, W2): W1 M(a1) + W2 M(a2) = I for the four invariants
    double x[4] = {0.1, 0.45, 0.05, 0.11}, I[4];
    invariant_integrals(I);
    for (int it = 0; it < 50; it++) {
        double m1[4], dm1[4], m2[4], dm2[4], F[4], J[4][4];
        orbit_moments(x[0], m1, dm1);
        orbit_moments(x[1], m2, dm2);
        double nrm = 0.0;
        for (int k = 0; k < 4; k++) {
            F[k] = x[2] * m1[k] + x[3] * m2[k] - I[k];
            nrm += std::fabs(F[k]);
            J[k][0] = x[2] * dm1[k];
            J[k][1] = x[3] * dm2[k];
            J[k][2] = m1[k];
            J[k][3] = m2[k];
        }
        if (nrm < 1e-17) break;
        // solve J dx = -F by Gaussian elimination with partial pivoting
        double A[4][5];
        for (int k = 0; k < 4; k++) {
            for (int c = 0; c < 4; c++) A[k][c] = J[k][c];
            A[k][4] = -F[k];
        }
        for (int c = 0; c < 4; c++) {
            int piv = c;
            for (int r = c + 1; r < 4; r++)
                if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
            for (int k = 0; k < 5; k++) std::swap(A[c][k], A[piv][k]);
            for (int r = c + 1; r < 4; r++) {
                const double f = A[r][c] / A[c][c];
                for (int k = c; k < 5; k++) A[r][k] -= f * A[c][k];
            }
        }
        double dx[4];
        for (int c = 3; c >= 0; c--) {
            double t = A[c][4];
            for (int k = c + 1; k < 4; k++) t -= A[c][k] * dx[k];
            dx[c] = t / A[c][c];
        }
        for (int c = 0; c < 4; c++) x[c] += dx[c];
    }
    const double a[2] = {x[0], x[1]};
    for (int o = 0; o < 2; o++) {
        const double pts[3][2] = {{a[o], a[o]}, {1.0 - 2.0 * a[o], a[o]}, {a[o], 1.0 - 2.0 * a[o]}};
        for (int i = 0; i < 3; i++) {
            rs[3 * o + i][0] = pts[i][0];
            rs[3 * o + i][1] = pts[i][1];
            w[3 * o + i] = x[2 + o];
        }
    }
    return true;
}

// Homogeneous barycentric monomials l1^i l2^j l3^k, i + j + k = p: a basis of the degree-p
// polynomials on the triangle.  Value and (r, s) derivatives (dl1 = (-1, -1), dl2 = (1, 0),
// dl3 = (0, 1)).
int bary_exps(int p, int (*ex)[3])
{
    int n = 0;
    for (int i = p; i >= 0; i--)
        for (int j = p - i; j >= 0; j--) {
            ex[n][0] = i;
            ex[n][1] = j;
            ex[n][2] = p - i - j;
            n++;
        }
    return n;
}
void bary_eval(const int e[3], double r, double s, double& v, double& vr, double& vs)
{
    const double l[3] = {1.0 - r - s, r, s};
    const double dlr[3] = {-1.0, 1.0, 0.0}, dls[3] = {-1.0, 0.0, 1.0};
    double pw[3], dpw[3];
    for (int k = 0; k < 3; k++) {
        pw[k] = std::pow(l[k], e[k]);
        dpw[k] = e[k] > 0 ? e[k] * std::pow(l[k], e[k] - 1) : 0.0;
    }
    v = pw[0] * pw[1] * pw[2];
    vr = vs = 0.0;
    for (int k = 0; k < 3; k++) {
        const double rest = pw[(k + 1) % 3] * pw[(k + 2) % 3];
        vr += dpw[k] * dlr[k] * rest;
        vs += dpw[k] * dls[k] * rest;
    }
}

// Lagrange basis on the solution points: phi_j = sum_m c[m][j] b_m with the barycentric
// monomials b_m; c = V^-1 for V[i][m] = b_m(x_i), by LU factorisation (Doolittle, partial
// pivoting) and one solve per unit vector.
bool build_tri_ops(int p, const FrOps& gl, TriOps& o)
{
    if (p < 1 || p > TRI_PMAX) return false;
    std::memset(&o, 0, sizeof(o));
    o.p = p;
    o.ns = (p + 1) * (p + 2) / 2;
    o.nfp = 3 * (p + 1);
    double rs[TRI_NSMAX][2];
    if (!ws_points(p, rs, o.wq)) return false;
    int ex[TRI_NSMAX][3];
    const int n = bary_exps(p, ex);
    double LU[TRI_NSMAX][TRI_NSMAX];
    int perm[TRI_NSMAX];
    for (int i = 0; i < n; i++) {
        perm[i] = i;
        for (int m = 0; m < n; m++) {
            double v, vr, vs;
            bary_eval(ex[m], rs[i][0], rs[i][1], v, vr, vs);
            LU[i][m] = v;
        }
    }
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (std::fabs(LU[r][c]) > std::fabs(LU[piv][c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; k++) std::swap(LU[c][k], LU[piv][k]);
            std::swap(perm[c], perm[piv]);
        }
        for (int r = c + 1; r < n; r++) {
            LU[r][c] /= LU[c][c];
            for (int k = c + 1; k < n; k++) LU[r][k] -= LU[r][c] * LU[c][k];
        }
    }
    double cf[TRI_NSMAX][TRI_NSMAX];   // cf[m][j]
    for (int j = 0; j < n; j++) {
        double y[TRI_NSMAX];
        for (int i = 0; i < n; i++) {   // L y = P e_j
            double t = perm[i] == j ? 1.0 : 0.0;
            for (int k = 0; k < i; k++) t -= LU[i][k] * y[k];
            y[i] = t;
        }
        for (int i = n - 1; i >= 0; i--) {   // U c = y
            double t = y[i];
            for (int k = i + 1; k < n; k++) t -= LU[i][k] * cf[k][j];
            cf[i][j] = t / LU[i][i];
        }
    }
    auto phi = [&](int j, double r, double s, double& v, double& vr, double& vs) {
        v = vr = vs = 0.0;
        for (int m = 0; m < n; m++) {
            double b, br, bs;
            bary_eval(ex[m], r, s, b, br, bs);
            v += cf[m][j] * b;
            vr += cf[m][j] * br;
            vs += cf[m][j] * bs;
        }
    };
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double v, vr, vs;
            phi(j, rs[i][0], rs[i][1], v, vr, vs);
            o.dr[i][j] = vr;
            o.ds[i][j] = vs;
        }
    const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    for (int f = 0; f < 3; f++)
        for (int k = 0; k <= p; k++) {
            const double t = 0.5 * (1.0 + gl.x[k]);
            const double r = V[f][0] + t * (V[(f + 1) % 3][0] - V[f][0]);
            const double s = V[f][1] + t * (V[(f + 1) % 3][1] - V[f][1]);
            const int q = f * (p + 1) + k;
            o.gw[q] = gl.wq[k];
            for (int j = 0; j < n; j++) {
                double v, vr, vs;
                phi(j, r, s, v, vr, vs);
                o.phif[q][j] = v;
            }
        }
    for (int q = 0; q < o.nfp; q++)
        for (int i = 0; i < n; i++) o.lift[q][i] = o.phif[q][i] * o.gw[q] / (2.0 * o.wq[i]);
    for (int i = 0; i < TRI_NSMAX; i++)
        for (int j = 0; j < TRI_NSMAX; j++) {
            o.drf[i][j] = (float)o.dr[i][j];
            o.dsf[i][j] = (float)o.ds[i][j];
        }
    for (int q = 0; q < TRI_NFPMAX; q++)
        for (int j = 0; j < TRI_NSMAX; j++) {
            o.phiff[q][j] = (float)o.phif[q][j];
            o.liftf[q][j] = (float)o.lift[q][j];
        }
    return true;
}

// ---- device -----------------------------------------------------------------------
struct TriMeshDev {
    int E, p;
    const TriGeo* geo;
    const int* nbr;
    const int* nbr_edge;
    const double* bc;
    // curved elements: per solution point (adj J = |J| J^-1 row by row, |J|): pj[E][ns][5]; per
    // flux point (physical unit normal, stretch |dx/dt| / |dxi/dt|): fq[E][nfp][3]
    const double* pj;
    const double* fq;
};

__device__ __forceinline__ const double* tri_exterior(const TriMeshDev& m, const double* __restrict__ wf, int e,
                                                      int f, int k)
{
    const int nb = m.nbr[e * 3 + f];
    if (nb >= 0) return wf + ((size_t)nb * 3 * (m.p + 1) + m.nbr_edge[e * 3 + f] * (m.p + 1) + (m.p - k)) * 4;
    return m.bc + (size_t)(-nb - 1) * 4;
}

// NS: the solution points per element, fixed at compile time so that the sum unrolls whole (a
// run-time count leaves a remainder the compiler predicates, and FP64 instructions issued with
// every lane off still take the slow FP64 pipe)
template <int NS>
__global__ void k_tri_traces(const double* __restrict__ w, double* __restrict__ wf, int E, TriOps o)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)E * o.nfp) return;
    const int e = (int)(t / o.nfp), q = (int)(t % o.nfp);
    const double* we = w + (size_t)e * NS * 4;
#pragma unroll
    for (int v = 0; v < 4; v++) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NS; j++) s += o.phif[q][j] * we[j * 4 + v];
        wf[((size_t)e * o.nfp + q) * 4 + v] = s;
    }
}

__global__ void k_tri_gather(const double* __restrict__ w, const double* __restrict__ wf, TriMeshDev m, int ns,
                             int nfp, double* __restrict__ S)
{
    const int nst = ns + 2 * nfp;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)m.E * nst) return;
    const int e = (int)(t / nst), r = (int)(t % nst);
    const double* src;
    if (r < ns) src = w + ((size_t)e * ns + r) * 4;
    else if (r < ns + nfp) src = wf + ((size_t)e * nfp + (r - ns)) * 4;
    else {
        const int q = r - ns - nfp;
        src = tri_exterior(m, wf, e, q / (m.p + 1), q % (m.p + 1));
    }
    double* dst = S + ((size_t)e * nst + r) * 4;
    dst[0] = src[0];
    dst[1] = src[1];
    dst[2] = src[2];
    dst[3] = src[3];
}

// Common flux along the outward unit normal (nx, ny), interior state qi on the minus side: the
// configured 1D flux of the states rotated into the edge's (n, t) frame, rotated back.
template <typename T>
__device__ __forceinline__ void tri_common_flux(const T* qi, const T* qe, T nx, T ny, T gamma, int flux, T* F)
{
    const T li[4] = {qi[0], qi[1] * nx + qi[2] * ny, -qi[1] * ny + qi[2] * nx, qi[3]};
    const T le[4] = {qe[0], qe[1] * nx + qe[2] * ny, -qe[1] * ny + qe[2] * nx, qe[3]};
    T Fl[4];
    if (flux == 1) kbl_hllc<2, T>(li, le, 0, gamma, Fl);
    else if (flux == 2) kbl_hll<2, T>(li, le, 0, gamma, Fl);
    else kbl_rusanov<2, T>(li, le, 0, gamma, Fl);
    F[0] = Fl[0];
    F[1] = Fl[1] * nx - Fl[2] * ny;
    F[2] = Fl[1] * ny + Fl[2] * nx;
    F[3] = Fl[3];
}

template <typename T>
__device__ __forceinline__ T tri_in(double x) { return kbl_dev::from_f64<T>(x); }

// One thread per element, order P fixed at compile time (the loops unroll, the fluxes stay in
// registers), arithmetic T (FP64, or FP32 on FP64 storage for the mixed precision).  The
// physical fluxes enter as contravariant fluxes Fr = (dr/dx) Fx + (dr/dy) Fy, Fs = (ds/dx) Fx +
// (ds/dy) Fy, so that -div F_h(x_i) = -sum_j (dr_ij Fr_j + ds_ij Fs_j); the normal flux at a flux
// point is a_f Fr_h + b_f Fs_h with (a_f, b_f) = J^T n_f of its edge; the jump of the common flux
// is lifted with lift_qi |e_f| / det J.
template <int P, typename T>
__global__ void __launch_bounds__(128) k_tri_rhs(const double* __restrict__ w, const double* __restrict__ wf,
                                                 TriMeshDev m, TriOps o, double gamma_d, int flux,
                                                 double* __restrict__ R)
{
    constexpr bool F32 = sizeof(T) == sizeof(float);
    constexpr int ns = (P + 1) * (P + 2) / 2, nfp = 3 * (P + 1);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const TriGeo& g = m.geo[e];
    const T rx = tri_in<T>(g.rx), ry = tri_in<T>(g.ry), sx = tri_in<T>(g.sx), sy = tri_in<T>(g.sy);
    const T gamma = tri_in<T>(gamma_d), gm1 = F32 ? gamma - T(1) : tri_in<T>(gamma_d - 1.0);
    T Fr[ns][4], Fs[ns][4], out[ns][4];
#pragma unroll
    for (int j = 0; j < ns; j++) {
        T q[4], Fx[4], Fy[4];
#pragma unroll
        for (int v = 0; v < 4; v++) q[v] = tri_in<T>(w[((size_t)e * ns + j) * 4 + v]);
        kbl_flux<2, T>(q, 0, gm1, Fx);
        kbl_flux<2, T>(q, 1, gm1, Fy);
#pragma unroll
        for (int v = 0; v < 4; v++) {
            Fr[j][v] = rx * Fx[v] + ry * Fy[v];
            Fs[j][v] = sx * Fx[v] + sy * Fy[v];
        }
    }
#pragma unroll
    for (int i = 0; i < ns; i++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            T div = T(0);
#pragma unroll
            for (int j = 0; j < ns; j++) {
                const T dr = F32 ? (T)o.drf[i][j] : (T)o.dr[i][j];
                const T ds = F32 ? (T)o.dsf[i][j] : (T)o.ds[i][j];
                div += dr * Fr[j][v] + ds * Fs[j][v];
            }
            out[i][v] = -div;
        }
    // J = inverse of ((rx, ry), (sx, sy)): J00 = x_r = sy det, J01 = x_s = -ry det, J10 = y_r = -sx det,
    // J11 = y_s = rx det
    const T det = tri_in<T>(g.det);
#pragma unroll 1
    for (int f = 0; f < 3; f++) {
        const T nx = tri_in<T>(g.nx[f]), ny = tri_in<T>(g.ny[f]);
        const T a = det * (sy * nx - sx * ny), b = det * (rx * ny - ry * nx);
        const T sc = tri_in<T>(g.len[f]) / det;
#pragma unroll
        for (int k = 0; k <= P; k++) {
            const int q = f * (P + 1) + k;
            T qi[4], qe[4], Fc[4];
            const double* ext = tri_exterior(m, wf, e, f, k);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                qi[v] = tri_in<T>(wf[((size_t)e * nfp + q) * 4 + v]);
                qe[v] = tri_in<T>(ext[v]);
            }
            tri_common_flux<T>(qi, qe, nx, ny, gamma, flux, Fc);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                T fr = T(0), fs = T(0);
#pragma unroll
                for (int j = 0; j < ns; j++) {
                    const T ph = F32 ? (T)o.phiff[q][j] : (T)o.phif[q][j];
                    fr += ph * Fr[j][v];
                    fs += ph * Fs[j][v];
                }
                const T jump = sc * (Fc[v] - (a * fr + b * fs));
#pragma unroll
                for (int i = 0; i < ns; i++) out[i][v] -= (F32 ? (T)o.liftf[q][i] : (T)o.lift[q][i]) * jump;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ns; i++)
#pragma unroll
        for (int v = 0; v < 4; v++) R[((size_t)e * ns + i) * 4 + v] = kbl_dev::to_f64<T>(out[i][v]);
}

// The residual on curved elements (transformed-flux form): with adj J = |J| J^-1 at each
// solution point, Ft = adj J F; at each flux point the physical unit normal n and the stretch
// sigma = |dx/dt| / |dxi/dt| of its edge; nh the reference edge's unit normal, L its length:
//   R_i = -(1/|J_i|) [ sum_j (Dr_ij Ft_r,j + Ds_ij Ft_s,j)
//                      + sum_q phi_i(x_q) gw_q L / (2 w_i) (sigma_q F*_n,q - (Ft_h . nh)(x_q)) ].
// One thread per element, as the affine kernel.
template <int P, typename T>
__global__ void __launch_bounds__(128) k_tri_rhs_curved(const double* __restrict__ w, const double* __restrict__ wf,
                                                        TriMeshDev m, TriOps o, double gamma_d, int flux,
                                                        double* __restrict__ R)
{
    constexpr bool F32 = sizeof(T) == sizeof(float);
    constexpr int ns = (P + 1) * (P + 2) / 2, nfp = 3 * (P + 1);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const double* pj = m.pj + (size_t)e * ns * 5;
    const double* fq = m.fq + (size_t)e * nfp * 3;
    const T gamma = tri_in<T>(gamma_d), gm1 = F32 ? gamma - T(1) : tri_in<T>(gamma_d - 1.0);
    T Fr[ns][4], Fs[ns][4], acc[ns][4];
#pragma unroll
    for (int j = 0; j < ns; j++) {
        T q[4], Fx[4], Fy[4];
#pragma unroll
        for (int v = 0; v < 4; v++) q[v] = tri_in<T>(w[((size_t)e * ns + j) * 4 + v]);
        kbl_flux<2, T>(q, 0, gm1, Fx);
        kbl_flux<2, T>(q, 1, gm1, Fy);
        const T a0 = tri_in<T>(pj[j * 5 + 0]), a1 = tri_in<T>(pj[j * 5 + 1]);
        const T a2 = tri_in<T>(pj[j * 5 + 2]), a3 = tri_in<T>(pj[j * 5 + 3]);
#pragma unroll
        for (int v = 0; v < 4; v++) {
            Fr[j][v] = a0 * Fx[v] + a1 * Fy[v];
            Fs[j][v] = a2 * Fx[v] + a3 * Fy[v];
        }
    }
#pragma unroll
    for (int i = 0; i < ns; i++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            T div = T(0);
#pragma unroll
            for (int j = 0; j < ns; j++) {
                const T dr = F32 ? (T)o.drf[i][j] : (T)o.dr[i][j];
                const T ds = F32 ? (T)o.dsf[i][j] : (T)o.ds[i][j];
                div += dr * Fr[j][v] + ds * Fs[j][v];
            }
            acc[i][v] = div;
        }
#pragma unroll 1
    for (int f = 0; f < 3; f++) {
        // reference edges: (0,0)->(1,0), (1,0)->(0,1), (0,1)->(0,0); unit normals and lengths
        const T nhx = f == 0 ? T(0) : (f == 1 ? T(0.70710678118654752) : T(-1));
        const T nhy = f == 0 ? T(-1) : (f == 1 ? T(0.70710678118654752) : T(0));
        const T L = f == 1 ? T(1.4142135623730951) : T(1);
#pragma unroll
        for (int k = 0; k <= P; k++) {
            const int q = f * (P + 1) + k;
            const T nx = tri_in<T>(fq[q * 3 + 0]), ny = tri_in<T>(fq[q * 3 + 1]), sig = tri_in<T>(fq[q * 3 + 2]);
            T qi[4], qe[4], Fc[4];
            const double* ext = tri_exterior(m, wf, e, f, k);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                qi[v] = tri_in<T>(wf[((size_t)e * nfp + q) * 4 + v]);
                qe[v] = tri_in<T>(ext[v]);
            }
            tri_common_flux<T>(qi, qe, nx, ny, gamma, flux, Fc);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                T fr = T(0), fs = T(0);
#pragma unroll
                for (int j = 0; j < ns; j++) {
                    const T ph = F32 ? (T)o.phiff[q][j] : (T)o.phif[q][j];
                    fr += ph * Fr[j][v];
                    fs += ph * Fs[j][v];
                }
                const T jump = L * (sig * Fc[v] - (nhx * fr + nhy * fs));
#pragma unroll
                for (int i = 0; i < ns; i++) acc[i][v] += (F32 ? (T)o.liftf[q][i] : (T)o.lift[q][i]) * jump;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ns; i++) {
        const T det = tri_in<T>(pj[i * 5 + 4]);
#pragma unroll
        for (int v = 0; v < 4; v++) R[((size_t)e * ns + i) * 4 + v] = kbl_dev::to_f64<T>(-acc[i][v] / det);
    }
}

// SSP-RK3 combination (Shu-Osher form) and the traces of its result (k_tri_traces' arithmetic,
// in its order) in one pass: a block combines the values of 32 elements, keeps them in shared
// memory and interpolates them to the flux points.
template <int P>
__global__ void __launch_bounds__(256) k_tri_combine_traces(int s, const double* __restrict__ wn, const double* ws,
                                                           const double* __restrict__ R, double dt, double* wout,
                                                           double* __restrict__ wf, int E, TriOps o)
{
    constexpr int ns = (P + 1) * (P + 2) / 2, nfp = 3 * (P + 1), EPB = 32;
    __shared__ double sw[EPB * ns * 4];
    const int e0 = blockIdx.x * EPB;
    const int ne = min(EPB, E - e0);
    const size_t base = (size_t)e0 * ns * 4;
    for (int i = threadIdx.x; i < ne * ns * 4; i += blockDim.x) {
        const size_t t = base + i;
        const double v = ws[t] + dt * R[t];
        const double r = s == 0 ? v : (s == 1 ? 0.75 * wn[t] + 0.25 * v : (1.0 / 3.0) * wn[t] + (2.0 / 3.0) * v);
        wout[t] = r;
        sw[i] = r;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ne * nfp * 4; i += blockDim.x) {
        const int el = i / (nfp * 4), rem = i - el * (nfp * 4), q = rem >> 2, v = rem & 3;
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < ns; j++) acc += o.phif[q][j] * sw[(el * ns + j) * 4 + v];
        wf[(size_t)(e0 + el) * nfp * 4 + rem] = acc;
    }
}

// dt bits: min over elements and solution points of h / (|U| + c) (positive doubles order as their bits).
__global__ void k_tri_dt(const double* __restrict__ w, TriMeshDev m, int ns, double gamma,
                         unsigned long long* bits)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double best = DBL_MAX;
    if (e < m.E) {
        const double h = m.geo[e].h;
        for (int i = 0; i < ns; i++) {
            const double* q = w + ((size_t)e * ns + i) * 4;
            const double P = kbl_pressure<2, double>(q, gamma - 1.0);
            const double u = sqrt(q[1] * q[1] + q[2] * q[2]) / q[0];
            best = fmin(best, h / (u + sqrt(gamma * P / q[0])));
        }
    }
    unsigned long long b = __double_as_longlong(best);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
        b = ob < b ? ob : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(bits, b);
}

}  // namespace

struct kbl_tri {
    kbl_config cfg;
    kbl_ctx* ctx = nullptr;     // bounds of explicit stencils and node-set limiting
    TriOps ops;
    int E = 0, n_bc = 0;
    cudaStream_t stream = nullptr;
    TriGeo* d_geo = nullptr;
    bool curved = false;
    double* d_pj = nullptr;     // curved: [E][ns][5] adj J and |J| at the solution points
    double* d_fq = nullptr;     // curved: [E][nfp][3] unit normal and stretch at the flux points
    double* d_wlim = nullptr;   // curved: [E][ns] the limiter's mean weights w_i |J_i|
    int* d_nbr = nullptr;
    int* d_nbr_edge = nullptr;
    double* d_bc = nullptr;
    double *d_wf = nullptr, *d_bnd = nullptr, *d_R = nullptr, *d_wa = nullptr, *d_wb = nullptr;
    unsigned long long* d_bits = nullptr;
    // the residual's branch: it runs beside the bounds of the same stage (both read only the
    // stage input and its traces)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
};

namespace {

kbl_status tfail(kbl_tri* t, kbl_status st, const std::string& msg)
{
    if (t) t->err = msg;
    return st;
}

TriMeshDev tri_dev(const kbl_tri* t)
{
    TriMeshDev m;
    m.E = t->E;
    m.p = t->cfg.p;
    m.geo = t->d_geo;
    m.nbr = t->d_nbr;
    m.nbr_edge = t->d_nbr_edge;
    m.bc = t->d_bc;
    m.pj = t->d_pj;
    m.fq = t->d_fq;
    return m;
}

unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

extern "C" {

kbl_status kbl_tri_points(int p, double* rs, double* w)
{
    if (!rs || !w) return KBL_EINVAL;
    double pts[TRI_NSMAX][2], wq[TRI_NSMAX];
    if (!ws_points(p, pts, wq)) return KBL_EINVAL;
    const int ns = (p + 1) * (p + 2) / 2;
    for (int i = 0; i < ns; i++) {
        rs[2 * i] = pts[i][0];
        rs[2 * i + 1] = pts[i][1];
        w[i] = wq[i];
    }
    return KBL_OK;
}

kbl_status kbl_tri_destroy(kbl_tri* t)
{
    if (!t) return KBL_EINVAL;
    void* ptrs[] = {t->d_geo, t->d_nbr, t->d_nbr_edge, t->d_bc, t->d_wf,   t->d_bnd,  t->d_R,
                    t->d_wa,  t->d_wb,  t->d_bits,     t->d_pj, t->d_fq, t->d_wlim};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (t->ev_fork) cudaEventDestroy(t->ev_fork);
    if (t->ev_join) cudaEventDestroy(t->ev_join);
    if (t->side) cudaStreamDestroy(t->side);
    if (t->ctx) kbl_destroy(t->ctx);
    delete t;
    return KBL_OK;
}

}  // extern "C"

namespace {

// Derivatives x_r, x_s, y_r, y_s at (r, s) of the quadratic map of the six points X[6][2] (the
// corners, then the mid-parameter points of edges 0, 1, 2): with barycentrics b1 = 1 - r - s,
// b2 = r, b3 = s the shape functions are b1 (2 b1 - 1), b2 (2 b2 - 1), b3 (2 b3 - 1), 4 b1 b2,
// 4 b2 b3, 4 b3 b1.
void quad_map_deriv(const double* X, double r, double s, double d[4])
{
    const double b1 = 1.0 - r - s;
    const double gr[6] = {1.0 - 4.0 * b1, 4.0 * r - 1.0, 0.0, 4.0 * (b1 - r), 4.0 * s, -4.0 * s};
    const double gs[6] = {1.0 - 4.0 * b1, 0.0, 4.0 * s - 1.0, -4.0 * r, 4.0 * r, 4.0 * (b1 - s)};
    d[0] = d[1] = d[2] = d[3] = 0.0;
    for (int k = 0; k < 6; k++) {
        d[0] += gr[k] * X[2 * k];       // x_r
        d[1] += gs[k] * X[2 * k];       // x_s
        d[2] += gr[k] * X[2 * k + 1];   // y_r
        d[3] += gs[k] * X[2 * k + 1];   // y_s
    }
}

kbl_status tri_create(kbl_tri** out, const kbl_config* cfg, int n_elem, const double* xy, const double* xy6,
                      const int32_t* nbr, const int32_t* nbr_edge, int n_bc, const double* bc, void* cuda_stream)
{
    if (!out) return KBL_EINVAL;
    *out = nullptr;
    if (!kbl_config_valid(cfg) || cfg->dim != 2 || cfg->p < 1 || cfg->p > TRI_PMAX) return KBL_EINVAL;
    if (n_elem < 0 || n_bc < 0 || (n_elem > 0 && (!xy || !nbr || !nbr_edge)) || (n_bc > 0 && !bc)) return KBL_EINVAL;
    for (long i = 0; i < 3L * n_elem; i++) {
        const int b = nbr[i], g = nbr_edge[i];
        if (b >= n_elem || (b < 0 && -(b + 1) >= n_bc) || (b >= 0 && (g < 0 || g > 2))) return KBL_EINVAL;
    }
    kbl_tri* t = new (std::nothrow) kbl_tri();
    if (!t) return KBL_ENOMEM;
    t->cfg = *cfg;
    t->E = n_elem;
    t->n_bc = n_bc;
    t->stream = (cudaStream_t)cuda_stream;
    kbl_status st = kbl_create(&t->ctx, cfg, cuda_stream);
    if (st != KBL_OK) {
        delete t;
        return st;
    }
    FrOps gl;
    kbl_build_fr_ops(cfg->p, gl);
    if (!build_tri_ops(cfg->p, gl, t->ops)) {
        kbl_tri_destroy(t);
        return KBL_EINVAL;
    }
    // geometry on the host
    std::vector<TriGeo> geo(std::max(1, n_elem));
    for (int e = 0; e < n_elem; e++) {
        const double* X = xy + (size_t)e * 6;
        const double J00 = X[2] - X[0], J10 = X[3] - X[1], J01 = X[4] - X[0], J11 = X[5] - X[1];
        TriGeo& g = geo[e];
        g.det = J00 * J11 - J01 * J10;
        if (!(g.det > 0.0)) {
            kbl_tri_destroy(t);
            return KBL_EINVAL;   // degenerate or clockwise element
        }
        g.rx = J11 / g.det;
        g.ry = -J01 / g.det;
        g.sx = -J10 / g.det;
        g.sy = J00 / g.det;
        double lmax = 0.0;
        for (int f = 0; f < 3; f++) {
            const double dx = X[2 * ((f + 1) % 3)] - X[2 * f], dy = X[2 * ((f + 1) % 3) + 1] - X[2 * f + 1];
            g.len[f] = std::sqrt(dx * dx + dy * dy);
            g.nx[f] = dy / g.len[f];
            g.ny[f] = -dx / g.len[f];
            lmax = std::max(lmax, g.len[f]);
        }
        g.h = g.det / lmax;
    }
    const size_t E = (size_t)std::max(1, n_elem), ns = t->ops.ns, nfp = t->ops.nfp;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
    };
    A((void**)&t->d_geo, E * sizeof(TriGeo));
    A((void**)&t->d_nbr, E * 3 * sizeof(int));
    A((void**)&t->d_nbr_edge, E * 3 * sizeof(int));
    A((void**)&t->d_bc, (size_t)std::max(1, n_bc) * 4 * sizeof(double));
    A((void**)&t->d_wf, E * nfp * 4 * sizeof(double));
    A((void**)&t->d_bnd, E * 8 * sizeof(double));
    A((void**)&t->d_R, E * ns * 4 * sizeof(double));
    A((void**)&t->d_wa, E * ns * 4 * sizeof(double));
    A((void**)&t->d_wb, E * ns * 4 * sizeof(double));
    A((void**)&t->d_bits, sizeof(unsigned long long));
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&t->side, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpy(t->d_geo, geo.data(), E * sizeof(TriGeo), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_elem > 0) e = cudaMemcpy(t->d_nbr, nbr, (size_t)n_elem * 3 * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_elem > 0)
        e = cudaMemcpy(t->d_nbr_edge, nbr_edge, (size_t)n_elem * 3 * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_bc > 0) e = cudaMemcpy(t->d_bc, bc, (size_t)n_bc * 4 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && xy6 && n_elem > 0) {
        // curved elements: metric terms at the solution points, normals and stretch at the
        // flux points, the limiter's mean weights
        double rs[TRI_NSMAX][2], wq[TRI_NSMAX];
        ws_points(cfg->p, rs, wq);
        const int p1 = cfg->p + 1;
        std::vector<double> pj((size_t)n_elem * ns * 5), fq((size_t)n_elem * nfp * 3), wl((size_t)n_elem * ns);
        const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
        bool ok = true;
        for (int el = 0; el < n_elem && ok; el++) {
            const double* X = xy6 + (size_t)el * 12;
            for (size_t i = 0; i < ns; i++) {
                double d[4];
                quad_map_deriv(X, rs[i][0], rs[i][1], d);
                const double det = d[0] * d[3] - d[1] * d[2];
                ok = ok && det > 0.0;
                double* o = &pj[((size_t)el * ns + i) * 5];
                o[0] = d[3];    // adj J = [[y_s, -x_s], [-y_r, x_r]]
                o[1] = -d[1];
                o[2] = -d[2];
                o[3] = d[0];
                o[4] = det;
                wl[(size_t)el * ns + i] = wq[i] * det;
            }
            for (int f = 0; f < 3; f++) {
                const double dvx = V[(f + 1) % 3][0] - V[f][0], dvy = V[(f + 1) % 3][1] - V[f][1];
                const double L = std::sqrt(dvx * dvx + dvy * dvy);
                for (int k = 0; k < p1; k++) {
                    const double tt = 0.5 * (1.0 + gl.x[k]);
                    double d[4];
                    quad_map_deriv(X, V[f][0] + tt * dvx, V[f][1] + tt * dvy, d);
                    const double tx = d[0] * dvx + d[1] * dvy, ty = d[2] * dvx + d[3] * dvy;
                    const double len = std::sqrt(tx * tx + ty * ty);
                    ok = ok && len > 0.0;
                    double* o = &fq[((size_t)el * nfp + f * p1 + k) * 3];
                    o[0] = ty / len;
                    o[1] = -tx / len;
                    o[2] = len / L;
                }
            }
        }
        if (!ok) {
            kbl_tri_destroy(t);
            return KBL_EINVAL;   // a folded or degenerate curved element
        }
        t->curved = true;
        A((void**)&t->d_pj, pj.size() * sizeof(double));
        A((void**)&t->d_fq, fq.size() * sizeof(double));
        A((void**)&t->d_wlim, wl.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(t->d_pj, pj.data(), pj.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(t->d_fq, fq.data(), fq.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(t->d_wlim, wl.data(), wl.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        kbl_tri_destroy(t);
        return e == cudaErrorMemoryAllocation ? KBL_ENOMEM : KBL_ECUDA;
    }
    *out = t;
    return KBL_OK;
}

}  // namespace

extern "C" {

kbl_status kbl_tri_create(kbl_tri** out, const kbl_config* cfg, int n_elem, const double* xy, const int32_t* nbr,
                          const int32_t* nbr_edge, int n_bc, const double* bc, void* cuda_stream)
{
    return tri_create(out, cfg, n_elem, xy, nullptr, nbr, nbr_edge, n_bc, bc, cuda_stream);
}

kbl_status kbl_tri_create_curved(kbl_tri** out, const kbl_config* cfg, int n_elem, const double* xy6,
                                 const int32_t* nbr, const int32_t* nbr_edge, int n_bc, const double* bc,
                                 void* cuda_stream)
{
    if (!out) return KBL_EINVAL;
    *out = nullptr;
    if (n_elem < 0 || (n_elem > 0 && !xy6)) return KBL_EINVAL;
    std::vector<double> corners((size_t)std::max(1, n_elem) * 6);
    for (long i = 0; i < (long)n_elem * 6; i++) corners[i] = xy6[(i / 6) * 12 + i % 6];
    return tri_create(out, cfg, n_elem, corners.data(), xy6, nbr, nbr_edge, n_bc, bc, cuda_stream);
}

const char* kbl_tri_last_error(const kbl_tri* t) { return t ? t->err.c_str() : "null triangle mesh"; }

kbl_status kbl_tri_traces(kbl_tri* t, const double* w, double* wf)
{
    if (!t || (t->E > 0 && (!w || !wf))) return tfail(t, KBL_EINVAL, "null array");
    const size_t n = (size_t)t->E * t->ops.nfp;
    if (n && t->ops.ns == 3) k_tri_traces<3><<<blocks_for(n, 256), 256, 0, t->stream>>>(w, wf, t->E, t->ops);
    else if (n) k_tri_traces<6><<<blocks_for(n, 256), 256, 0, t->stream>>>(w, wf, t->E, t->ops);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : tfail(t, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_tri_gather_stencil(kbl_tri* t, const double* w, const double* wf, double* S)
{
    if (!t || (t->E > 0 && (!w || !wf || !S))) return tfail(t, KBL_EINVAL, "null array");
    const size_t n = (size_t)t->E * (t->ops.ns + 2 * t->ops.nfp);
    if (n) k_tri_gather<<<blocks_for(n, 256), 256, 0, t->stream>>>(w, wf, tri_dev(t), t->ops.ns, t->ops.nfp, S);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : tfail(t, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_tri_bounds(kbl_tri* t, const double* w, const double* wf, double* bnd)
{
    if (!t || (t->E > 0 && (!w || !wf || !bnd))) return tfail(t, KBL_EINVAL, "null array");
    if (launch_bounds_tri(t->ctx, t->E, t->cfg.p, w, wf, t->d_nbr, t->d_nbr_edge, t->d_bc, bnd, t->stream) < 0)
        return tfail(t, KBL_EINVAL, "bounds of this order not compiled in");
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : tfail(t, KBL_ECUDA, cudaGetErrorString(e));
}

namespace {

// The residual of kbl_tri_residual on a given stream.
kbl_status tri_residual_on(kbl_tri* t, const double* w, const double* wf, double* R, cudaStream_t s)
{
    if (t->E) {
        const unsigned grid = blocks_for(t->E, 128);
        const bool f32 = t->cfg.precision == KBL_FP32_MIXED;
        const TriMeshDev md = tri_dev(t);
        const double gam = t->cfg.gamma;
        const int fl = t->cfg.flux;
        if (t->curved) {
            if (t->cfg.p == 1 && f32) k_tri_rhs_curved<1, float><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
            else if (t->cfg.p == 1) k_tri_rhs_curved<1, double><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
            else if (f32) k_tri_rhs_curved<2, float><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
            else k_tri_rhs_curved<2, double><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
        } else if (t->cfg.p == 1 && f32) {
            k_tri_rhs<1, float><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
        } else if (t->cfg.p == 1) {
            k_tri_rhs<1, double><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
        } else if (f32) {
            k_tri_rhs<2, float><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
        } else {
            k_tri_rhs<2, double><<<grid, 128, 0, s>>>(w, wf, md, t->ops, gam, fl, R);
        }
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : tfail(t, KBL_ECUDA, cudaGetErrorString(e));
}

}  // namespace

kbl_status kbl_tri_residual(kbl_tri* t, const double* w, const double* wf, double* R)
{
    if (!t || (t->E > 0 && (!w || !wf || !R))) return tfail(t, KBL_EINVAL, "null array");
    return tri_residual_on(t, w, wf, R, t->stream);
}

kbl_status kbl_tri_dt(kbl_tri* t, const double* w, double cfl, double* dt_host)
{
    if (!t || !dt_host || !(cfl > 0.0) || (t->E > 0 && !w)) return tfail(t, KBL_EINVAL, "bad argument");
    *dt_host = 0.0;
    if (t->E == 0) return KBL_OK;
    cudaError_t e = cudaMemsetAsync(t->d_bits, 0x7f, sizeof(unsigned long long), t->stream);
    if (e == cudaSuccess)
        k_tri_dt<<<blocks_for(t->E, 128), 128, 0, t->stream>>>(w, tri_dev(t), t->ops.ns, t->cfg.gamma, t->d_bits);
    unsigned long long b = 0;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&b, t->d_bits, sizeof(b), cudaMemcpyDeviceToHost, t->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
    if (e != cudaSuccess) return tfail(t, KBL_ECUDA, cudaGetErrorString(e));
    double h;
    std::memcpy(&h, &b, sizeof(h));
    *dt_host = (h > 0.0 && h < 1e300) ? cfl * h : 0.0;   // 0 when no point gave a finite rate
    return KBL_OK;
}

// One SSP-RK3 step with a given dt: per stage the kinetic bounds of every stencil of the stage
// input (gathered inside the bounds kernel from the state and its traces; the configured
// precision and quadrature), the residual (on a side stream, beside the bounds), the combination, the traces of the combined state
// and the node-set limiter (the mean weights = the Williams-Shunn weights), which also writes the
// limited face values: the traces of the next stage's input.
kbl_status kbl_tri_step(kbl_tri* t, double* w, double dt)
{
    if (!t || (t->E > 0 && !w) || !(dt >= 0.0)) return tfail(t, KBL_EINVAL, "bad argument");
    if (t->E == 0) return KBL_OK;
    const int ns = t->ops.ns, nfp = t->ops.nfp;
    const double* ws = w;
    double* outs[3] = {t->d_wa, t->d_wb, w};
    kbl_status st;
    if ((st = kbl_tri_traces(t, w, t->d_wf)) != KBL_OK) return st;
    for (int s = 0; s < 3; s++) {
        // the residual on the side stream, beside the bounds; the combination waits for both
        cudaError_t ce = cudaEventRecord(t->ev_fork, t->stream);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(t->side, t->ev_fork, 0);
        if (ce != cudaSuccess) return tfail(t, KBL_ECUDA, cudaGetErrorString(ce));
        if ((st = tri_residual_on(t, ws, t->d_wf, t->d_R, t->side)) != KBL_OK) return st;
        ce = cudaEventRecord(t->ev_join, t->side);
        if (ce != cudaSuccess) return tfail(t, KBL_ECUDA, cudaGetErrorString(ce));
        if ((st = kbl_tri_bounds(t, ws, t->d_wf, t->d_bnd)) != KBL_OK) return st;
        ce = cudaStreamWaitEvent(t->stream, t->ev_join, 0);
        if (ce != cudaSuccess) return tfail(t, KBL_ECUDA, cudaGetErrorString(ce));
        const unsigned gct = blocks_for((size_t)t->E, 32);
        if (t->cfg.p == 1)
            k_tri_combine_traces<1><<<gct, 256, 0, t->stream>>>(s, w, ws, t->d_R, dt, outs[s], t->d_wf, t->E, t->ops);
        else
            k_tri_combine_traces<2><<<gct, 256, 0, t->stream>>>(s, w, ws, t->d_R, dt, outs[s], t->d_wf, t->E, t->ops);
        launch_limit_nodes(t->ctx, t->E, ns, nfp, t->ops.wq, outs[s], t->d_wf, t->d_bnd, nullptr, t->stream,
                           t->d_wf, t->curved ? t->d_wlim : nullptr);
        ws = outs[s];
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : tfail(t, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_tri_check(kbl_tri* t)
{
    if (!t) return KBL_EINVAL;
    const kbl_status st = kbl_check(t->ctx);
    return st == KBL_OK ? KBL_OK : tfail(t, st, kbl_last_error(t->ctx));
}

}  // extern "C"
