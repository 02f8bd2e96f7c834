// kbl_adjoint_body.cuh -- vector-Jacobian products (reverse-mode derivatives) of the
// Euler physics used by the FR residual and the kinetic bounds, FP64.
//
// Conventions: q = (rho, m_x[, m_y], E); every *_vjp adds to its output cotangents.
#pragma once

#include "kbl_internal.cuh"

namespace kbl_dev {

// qb += (dF_D/dq)^T Fb for the Euler flux along axis D (Eq. 2).
//   dP/drho = (g-1)|u|^2/2, dP/dm_l = -(g-1) u_l, dP/dE = g-1
//   F_0 = m_D
//   F_{1+k} = m_k u_D + P delta_kD
//   F_last = (E + P) u_D,  H = (E + P) / rho
// The axis is a template parameter: every index into the state is a compile-time
// constant.
template <int DIM, int D>
__device__ __forceinline__ void flux_vjp(const double* q, double gamma, const double* Fb, double* qb)
{
    const double gm1 = gamma - 1.0;
    const double rho = q[0], inv = 1.0 / rho;
    const double u0 = q[1] * inv, u1 = DIM == 2 ? q[2] * inv : 0.0;
    const double uu = u0 * u0 + u1 * u1;
    const double E = q[DIM + 1];
    const double P = gm1 * (E - 0.5 * rho * uu);
    const double H = (E + P) * inv;
    const double ud = D == 0 ? u0 : u1;
    // F_0 = m_D
    qb[1 + D] += Fb[0];
#pragma unroll
    for (int k = 0; k < DIM; k++) {
        const double fb = Fb[1 + k];
        const double uk = k == 0 ? u0 : u1;
        qb[0] += fb * (-uk * ud + (k == D ? 0.5 * gm1 * uu : 0.0));
#pragma unroll
        for (int l = 0; l < DIM; l++) {
            const double ul = l == 0 ? u0 : u1;
            const double dv = (k == l ? ud : 0.0) + (l == D ? uk : 0.0) - (k == D ? gm1 * ul : 0.0);
            qb[1 + l] += fb * dv;
        }
        if (k == D) qb[DIM + 1] += fb * gm1;
    }
    // energy row
    const double fe = Fb[DIM + 1];
    qb[0] += fe * ud * (0.5 * gm1 * uu - H);
#pragma unroll
    for (int l = 0; l < DIM; l++) {
        const double ul = l == 0 ? u0 : u1;
        qb[1 + l] += fe * (-gm1 * ul * ud + (l == D ? H : 0.0));
    }
    qb[DIM + 1] += fe * gamma * ud;
}

// Davis wavespeed |u_D| + c of one state, c = sqrt(gamma P / rho) (the forward expression).
template <int DIM, int D>
__device__ __forceinline__ double wavespeed(const double* q, double gamma)
{
    return fabs(q[1 + D] / q[0]) + sqrt(gamma * kbl_pressure<DIM>(q, gamma - 1.0) / q[0]);
}

// qb += sb * d(|u_D| + c)/dq; u_D = 0 takes the + branch.
template <int DIM, int D>
__device__ __forceinline__ void wavespeed_vjp(const double* q, double gamma, double sb, double* qb)
{
    const double gm1 = gamma - 1.0;
    const double rho = q[0], inv = 1.0 / rho;
    const double u0 = q[1] * inv, u1 = DIM == 2 ? q[2] * inv : 0.0;
    const double uu = u0 * u0 + u1 * u1;
    const double P = gm1 * (q[DIM + 1] - 0.5 * rho * uu);
    const double c = sqrt(gamma * P * inv);
    const double ud = D == 0 ? u0 : u1;
    const double sgn = ud < 0.0 ? -1.0 : 1.0;
    // |u_D|
    qb[0] += sb * sgn * (-ud * inv);
    qb[1 + D] += sb * sgn * inv;
    // c: dc = gamma / (2 c rho) (dP - P/rho drho)
    const double f = sb * gamma / (2.0 * c * rho);
    qb[0] += f * (0.5 * gm1 * uu - P * inv);
    qb[1] += f * (-gm1 * u0);
    if (DIM == 2) qb[2] += f * (-gm1 * u1);
    qb[DIM + 1] += f * gm1;
}

// Rusanov flux F = 1/2 (F(ql) + F(qr)) - 1/2 lam (qr - ql), lam = max(s_l, s_r) (Davis):
// qlb, qrb += its transposed Jacobian applied to Fb.  Ties of the max take the left state.
template <int DIM, int D>
__device__ __forceinline__ void rusanov_vjp(const double* ql, const double* qr, double gamma, const double* Fb,
                                            double* qlb, double* qrb)
{
    constexpr int NV = DIM + 2;
    const double sl = wavespeed<DIM, D>(ql, gamma);
    const double sr = wavespeed<DIM, D>(qr, gamma);
    const double lam = fmax(sl, sr);
    double half[NV], lamb = 0.0;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        half[v] = 0.5 * Fb[v];
        qrb[v] += -0.5 * lam * Fb[v];
        qlb[v] += 0.5 * lam * Fb[v];
        lamb += -0.5 * (qr[v] - ql[v]) * Fb[v];
    }
    flux_vjp<DIM, D>(ql, gamma, half, qlb);
    flux_vjp<DIM, D>(qr, gamma, half, qrb);
    if (sl >= sr) wavespeed_vjp<DIM, D>(ql, gamma, lamb, qlb);
    else wavespeed_vjp<DIM, D>(qr, gamma, lamb, qrb);
}

// qb += Pb * dP/dq, P = (gamma - 1)(E - |m|^2 / (2 rho)).
template <int DIM>
__device__ __forceinline__ void pressure_vjp(const double* q, double gamma, double Pb, double* qb)
{
    const double gm1 = gamma - 1.0;
    const double inv = 1.0 / q[0];
    const double u0 = q[1] * inv, u1 = DIM == 2 ? q[2] * inv : 0.0;
    qb[0] += Pb * gm1 * 0.5 * (u0 * u0 + u1 * u1);
    qb[1] += Pb * (-gm1 * u0);
    if (DIM == 2) qb[2] += Pb * (-gm1 * u1);
    qb[DIM + 1] += Pb * gm1;
}

}  // namespace kbl_dev
