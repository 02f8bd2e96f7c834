// kbl_limit.cu -- SSP-RK3 stage combination fused with the kinetic-bounds
// limiter (Sec. 3.4 and Sec. 3.8 of the paper), FP64.
//
// Per element, one thread per solution point:
//   w    = a_s wn + b_s (ws + dt R)            (Shu-Osher SSP-RK3; skipped in
//                                               limiter-only mode)
//   mean = sum W_n w_n / sum W_n               (Gauss-Legendre weights, Eq. 13)
//   face values by interpolation; V = solution points + face points
//   alpha_i  (Eq. 37 with the epsilon rule), alpha = min_i alpha_i (Eq. 39)
//   w~ = mean + alpha (w - mean) at solution and face points (Eq. 38)
//   P_min over V (Eq. 47); if < p_floor:
//     alpha_P = |(p_floor - P(mean)) / (P_min - P(mean))| (0 if P(mean) <= p_floor)
//     w~~ = mean + alpha_P (w~ - mean)          (Eq. 48-49)
#include <cfloat>

#include "kbl_limit_body.cuh"

namespace {

template <int DIM, int N>
struct LimShape {
    static constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    static constexpr int EPB = (DIM == 1) ? 32 : 8;
    static constexpr int NT = EPB * NS;
};

template <int DIM, int N>
__global__ void __launch_bounds__(LimShape<DIM, N>::NT)
k_stage_limit(int mode, int stage, const double* wn, const double* ws, const double* __restrict__ R,
              const double* __restrict__ bnd, const double* __restrict__ dtp, double* wout,
              double* __restrict__ alpha_out, int E, FrOps ops, Phys ph, DevFlags* flags)
{
    using SH = LimShape<DIM, N>;
    __shared__ kbl_dev::LimSmem<DIM, N, SH::EPB> sm;
    const double dt = (mode == 0) ? dtp[0] : 0.0;
    kbl_dev::stage_limit_block<DIM, N, SH::EPB>(sm, SH::NT, mode, stage, wn, ws, R, bnd, dt, wout, alpha_out, E,
                                                ops, ph, flags, blockIdx.x * SH::EPB, SH::EPB);
}

template <int DIM, int N>
int run_stage(const kbl_ctx* c, int mode, int stage, const double* wn, const double* ws,
              const double* R, const double* bnd, const double* dt, double* wout, double* alpha,
              cudaStream_t s)
{
    using SH = LimShape<DIM, N>;
    if (c->E == 0) return 0;
    const unsigned grid = (unsigned)((c->E + SH::EPB - 1) / SH::EPB);
    k_stage_limit<DIM, N><<<grid, SH::NT, 0, s>>>(mode, stage, wn, ws, R, bnd, dt, wout, alpha, c->E,
                                                 c->ops, c->phys, c->d_flags);
    return 1;
}

}  // namespace

int launch_stage(const kbl_ctx* c, int mode, int stage, const double* wn, const double* ws,
                 const double* R, const double* bnd, const double* dt, double* wout, double* alpha,
                 cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_stage, c, mode, stage, wn, ws, R, bnd, dt, wout, alpha, s);
}
