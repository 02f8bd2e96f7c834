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
// An exact FP32 screen (kbl_limit_body.cuh) first certifies, where it can, that alpha = 1
// and that no point of V fails the pressure test; those elements keep w and skip the FP64
// steps above, whose results they would not change beyond the rounding of mean + (w - mean).
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

// The stage kernel of kbl_step: the stage and limiter, then (wf_next) the next stage's face traces
// from the limited state still in shared memory, or (advance) the clock of the step.
#ifdef KBL_STAGE_MINB
#define KBL_STAGE_BOUNDS(...) __launch_bounds__(__VA_ARGS__, KBL_STAGE_MINB)
#else
#define KBL_STAGE_BOUNDS(...) __launch_bounds__(__VA_ARGS__)
#endif
template <int DIM, int N, int STAGE>
__global__ void KBL_STAGE_BOUNDS(LimShape<DIM, N>::NT)
k_stage_limit_step(const double* wn, const double* ws, const double* __restrict__ R,
                   const double* __restrict__ bnd, double* scal, double* wout, double* __restrict__ wf_next,
                   int advance, int E, FrOps ops, Phys ph, DevFlags* flags)
{
    using SH = LimShape<DIM, N>;
    // a programmatic dependent of the bounds launch: the stage combination and the screen's first
    // phases read only what was complete before that launch began (wn, ws, R, dt), so they run
    // while its last blocks finish; the body waits for it before its first read of the bounds
    kbl_grid_dep_trigger();
    __shared__ kbl_dev::LimSmem<DIM, N, SH::EPB> sm;
    const double dt = scal[0];
    const int e0 = blockIdx.x * SH::EPB;
    kbl_dev::stage_limit_block<DIM, N, SH::EPB, true, STAGE>(sm, SH::NT, 0, STAGE, wn, ws, R, bnd, dt, wout, nullptr,
                                                             E, ops, ph, flags, e0, SH::EPB);
    if (wf_next) kbl_dev::traces_of_block<DIM, N, SH::EPB>(sm, SH::NT, E, e0, SH::EPB, wf_next);
    // the clock: t += dt, once (no block of this launch reads t)
    if (advance && blockIdx.x == 0 && threadIdx.x == 0) scal[1] += dt;
}

template <int DIM, int N>
int run_stage_step(const kbl_ctx* c, int stage, const double* wn, const double* ws, const double* R, const double* bnd,
                   double* wout, double* wf_next, int advance, cudaStream_t s)
{
    using SH = LimShape<DIM, N>;
    if (c->E == 0) return 0;
    const unsigned grid = (unsigned)((c->E + SH::EPB - 1) / SH::EPB);
    // one kernel per stage: the stage's combination is fixed at compile time
    if (stage == 0)
        kbl_launch(k_stage_limit_step<DIM, N, 0>, grid, SH::NT, 0, s, c->pdl, wn, ws, R, bnd, c->d_scal, wout, wf_next,
                   advance, c->E, c->ops, c->phys, c->d_flags);
    else if (stage == 1)
        kbl_launch(k_stage_limit_step<DIM, N, 1>, grid, SH::NT, 0, s, c->pdl, wn, ws, R, bnd, c->d_scal, wout, wf_next,
                   advance, c->E, c->ops, c->phys, c->d_flags);
    else
        kbl_launch(k_stage_limit_step<DIM, N, 2>, grid, SH::NT, 0, s, c->pdl, wn, ws, R, bnd, c->d_scal, wout, wf_next,
                   advance, c->E, c->ops, c->phys, c->d_flags);
    return 1;
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

// ---------------------------------------------------------------------------
// Limiting of caller-assembled node sets (Eq. 37-39, Eq. 47-49), FP64, one thread per
// element: solution values U[E][ns][nv] (limited in place) with positive mean weights
// W[ns], face values F[E][nf][nv] (read only: they enter the extremes over V and the
// pressure minimum), bounds bnd[2][nv][E].  The operations and their order follow the FR
// limiter's exact path.
// ---------------------------------------------------------------------------
struct NodeWeights {
    double w[64];
};

// The node-set limiter, one thread per element, FP64 and the checker's arithmetic; three
// shortcuts leave every result as it is:
// - extrema of V through order-preserving integer keys (the integer pipe, not FP64 min/max);
// - Eq. 37 without its divisions when lo <= mn < mean < mx <= hi for the extremes mn, mx of V
//   (then both ratios are >= 1 after rounding: hi - mean >= mx - mean > 0 and
//   lo - mean <= mn - mean < 0 round monotonically), so alpha_i = 1;
// - the pressure test of Eq. 47 without divisions: gm1 (E rho - |m|^2 / 2) >= p_floor rho plus a
//   margin of 16 ulp of the terms proves P >= p_floor as the exact formula rounds it; only an
//   element that fails this test forms P_min with the divisions.
// - where alpha = 1 for every component, Eq. 47 screened in FP32 (below) and the values kept.
// We (may be NULL): per-element mean weights We[E][ns] in place of W (curved elements: w_i |J_i|).
// F_out (may be NULL; may alias F): the limited face values mean + alpha (f - mean), then the
// pressure step, as for the solution values: the traces of the limited state, whose
// interpolation weights sum to one.
template <int NV>
__global__ void __launch_bounds__(128) k_limit_nodes(int E, int ns, int nf, NodeWeights W, double* __restrict__ U,
                                                     const double* F, const double* __restrict__ bnd,
                                                     double* __restrict__ alpha_out, Phys ph, DevFlags* flags,
                                                     double* F_out, const double* __restrict__ We)
{
    constexpr int DIM = NV - 2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double* u = U + (size_t)e * ns * NV;
    const double* f = F + (size_t)e * nf * NV;
    const double* we = We ? We + (size_t)e * ns : nullptr;   // per-element mean weights, if given
    double mean[NV], av[NV], alpha = 1.0;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        double s = 0.0, sw = 0.0;
        for (int n = 0; n < ns; n++) {
            const double wn = we ? we[n] : W.w[n];
            s += wn * u[n * NV + v];
            sw += wn;
        }
        mean[v] = s / sw;
        long long kmx = kbl_dev::dkey(u[v]), kmn = kmx;
        for (int n = 1; n < ns; n++) {
            const long long k = kbl_dev::dkey(u[n * NV + v]);
            kmx = k > kmx ? k : kmx;
            kmn = k < kmn ? k : kmn;
        }
        for (int n = 0; n < nf; n++) {
            const long long k = kbl_dev::dkey(f[n * NV + v]);
            kmx = k > kmx ? k : kmx;
            kmn = k < kmn ? k : kmn;
        }
        const double mx = kbl_dev::dunkey(kmx), mn = kbl_dev::dunkey(kmn);
        const double dmax = mx - mean[v], dmin = mn - mean[v];
        const double lo = bnd[(size_t)v * E + e], hi = bnd[((size_t)NV + v) * E + e];
        if (mean[v] < lo || mean[v] > hi) atomicAdd(&flags->mean_outside, 1ull);
        double a;
        if (fabs(dmin) < ph.eps || fabs(dmax) < ph.eps) {
            atomicAdd(&flags->eps_rule, 1ull);
            a = ph.eps_rule ? 1.0 : 0.0;
        } else if (mx <= hi && mn >= lo && dmax > 0.0 && dmin < 0.0) {
            a = 1.0;
        } else {
            a = 1.0;
            const double t1 = fabs((hi - mean[v]) / dmax), t2 = fabs((lo - mean[v]) / dmin);
            if (t1 < a) a = t1;
            if (t2 < a) a = t2;
        }
        av[v] = a;
        if (a < alpha) alpha = a;
    }
    if (!ph.uncoupled)
#pragma unroll
        for (int v = 0; v < NV; v++) av[v] = alpha;
    const double gm1 = ph.gamma - 1.0;
    // alpha = 1 for every component (the common case): V limited is mean + (x - mean) = x up to
    // FP64 rounding of |x| + |mean|.  Screen Eq. 47 in FP32 on the truncated x: with A_v =
    // |x_v| + |mean_v|, the FP32 value of (gamma - 1)(E rho - |m|^2 / 2) differs from the FP64
    // one of the limited state by at most 2^-19 (gamma - 1)(A_E A_rho + A_m^2) (inputs truncated
    // to 2^-23, the limited state within 2^-52 A of x, a few FP32 roundings); a margin of 2^-16
    // of that, plus 2^-16 p_floor A_rho for the density's own error, then proves P >= p_floor as
    // the exact formula rounds it.  Magnitudes are held inside [2^-40, 2^40] so that nothing
    // overflows or loses its terms to underflow.  Such an element keeps its values (the FP64
    // mean + (x - mean) would move them by rounding only) and skips the FP64 steps below.
    if (alpha == 1.0) {
        float mf[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) mf[v] = fabsf(f32_trunc(mean[v]));
        const float gf = f32_trunc(gm1), pf = f32_trunc(ph.p_floor) * (1.0f + 0x1p-20f);
        bool ok = true;
        for (int n = 0; n < ns + nf && ok; n++) {
            const double* x = n < ns ? u + n * NV : f + (n - ns) * NV;
            float q[NV], A[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                q[v] = f32_trunc(x[v]);
                A[v] = fabsf(q[v]) + mf[v];
            }
            float mm = q[1] * q[1], am = A[1] * A[1];
            if (DIM == 2) {
                mm += q[2] * q[2];
                am += A[2] * A[2];
            }
            const float X = gf * (q[DIM + 1] * q[0] - 0.5f * mm);
            const float margin = 0x1p-16f * gf * (A[DIM + 1] * A[0] + am) + 0x1p-16f * pf * A[0];
            bool in_range = q[0] > 0x1p-40f && q[0] > 0x1p-10f * A[0] && A[DIM + 1] > 0x1p-40f;
#pragma unroll
            for (int v = 0; v < NV; v++) in_range = in_range && A[v] < 0x1p40f;
            ok = in_range && X >= pf * q[0] + margin;
        }
        if (ok) {
            if (F_out && F_out != F) {
                double* fo = F_out + (size_t)e * nf * NV;
                for (int n = 0; n < nf * NV; n++) fo[n] = f[n];
            }
            if (alpha_out) {
                alpha_out[e] = 1.0;
                alpha_out[(size_t)E + e] = 1.0;
            }
            return;
        }
    }
    // Eq. 47 over V of the limited values: first without divisions
    bool sure = true;
    for (int n = 0; n < ns + nf && sure; n++) {
        const double* x = n < ns ? u + n * NV : f + (n - ns) * NV;
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) q[v] = mean[v] + av[v] * (x[v] - mean[v]);
        double mm = q[1] * q[1];
        if (DIM == 2) mm += q[2] * q[2];
        const double er = q[DIM + 1] * q[0], hm = 0.5 * mm;
        const double margin = 16.0 * DBL_EPSILON * gm1 * (fabs(er) + hm) + 16.0 * DBL_EPSILON * ph.p_floor * q[0];
        sure = q[0] > 0.0 && gm1 * (er - hm) >= ph.p_floor * q[0] + margin;
    }
    double aP = 1.0;
    bool relimit = false;
    if (!sure) {
        double pmin = INFINITY;
        for (int n = 0; n < ns + nf; n++) {
            const double* x = n < ns ? u + n * NV : f + (n - ns) * NV;
            double q[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) q[v] = mean[v] + av[v] * (x[v] - mean[v]);
            pmin = fmin(pmin, kbl_pressure<DIM>(q, gm1));
        }
        relimit = pmin < ph.p_floor;
        if (relimit) {
            const double Pbar = kbl_pressure<DIM>(mean, gm1);
            aP = (Pbar > ph.p_floor) ? fabs((ph.p_floor - Pbar) / (pmin - Pbar)) : 0.0;
        }
    }
    if (F_out) {
        double* fo = F_out + (size_t)e * nf * NV;
        for (int n = 0; n < nf; n++)
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const double ft = mean[v] + av[v] * (f[n * NV + v] - mean[v]);
                fo[n * NV + v] = relimit ? mean[v] + aP * (ft - mean[v]) : ft;
            }
    }
    for (int n = 0; n < ns; n++)
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double wt = mean[v] + av[v] * (u[n * NV + v] - mean[v]);
            u[n * NV + v] = relimit ? mean[v] + aP * (wt - mean[v]) : wt;
        }
    if (alpha_out) {
        alpha_out[e] = alpha;
        alpha_out[(size_t)E + e] = aP;
    }
    if (alpha < 1.0) {
        atomicAdd(&flags->limited, 1ull);
        atomicAdd(&flags->alpha_hist[kbl_alpha_bin(alpha)], 1ull);
    }
    if (relimit) atomicAdd(&flags->prelimit, 1ull);
}

}  // namespace

int launch_limit_nodes(const kbl_ctx* c, int E, int ns, int nf, const double* W, double* U, const double* F,
                       const double* bnd, double* alpha, cudaStream_t s, double* F_out, const double* We)
{
    if (E == 0) return 0;
    NodeWeights nw;
    for (int n = 0; n < 64; n++) nw.w[n] = n < ns ? W[n] : 0.0;
    const unsigned grid = (unsigned)((E + 127) / 128);
    if (c->cfg.dim == 2)
        k_limit_nodes<4><<<grid, 128, 0, s>>>(E, ns, nf, nw, U, F, bnd, alpha, c->phys, c->d_flags, F_out, We);
    else
        k_limit_nodes<3><<<grid, 128, 0, s>>>(E, ns, nf, nw, U, F, bnd, alpha, c->phys, c->d_flags, F_out, We);
    return 1;
}

int launch_stage(const kbl_ctx* c, int mode, int stage, const double* wn, const double* ws,
                 const double* R, const double* bnd, const double* dt, double* wout, double* alpha,
                 cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_stage, c, mode, stage, wn, ws, R, bnd, dt, wout, alpha, s);
}

int launch_stage_step(const kbl_ctx* c, int stage, const double* wn, const double* ws, const double* R,
                      const double* bnd, double* wout, double* wf_next, int advance, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_stage_step, c, stage, wn, ws, R, bnd, wout, wf_next, advance, s);
}
