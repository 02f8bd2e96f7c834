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

#include "kbl_internal.cuh"

namespace {

// Order-preserving map of a double to a signed 64-bit key (finite values):
// min/max then run on the integer pipe instead of the slow FP64 pipe.
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double dunkey(long long k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

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
    constexpr int NS = SH::NS, NFP = SH::NFP, NV = SH::NV, EPB = SH::EPB, NT = SH::NT;
    constexpr int NFPF = (DIM == 1) ? 1 : N;
    __shared__ double sw[EPB][NV][NS];      // state at solution points (then limited)
    __shared__ double sf[EPB][NV][NFP];     // state at face points (then limited)
    __shared__ double smean[EPB][NV];
    __shared__ double salpha_v[EPB][NV];
    __shared__ double salpha[EPB];
    __shared__ double sP[EPB][NS + NFP];
    __shared__ double saP[EPB];
    __shared__ int sPtaken[EPB];
    __shared__ double slm[N], slp[N], sW[NS];
    __shared__ double sWsum;

    const int tid = threadIdx.x;
    if (tid < N) {
        slm[tid] = ops.lm[tid];
        slp[tid] = ops.lp[tid];
    }
    if (tid < NS) sW[tid] = (DIM == 1) ? ops.wq[tid] : ops.wq[tid % N] * ops.wq[tid / N];
    if (tid == 0) {
        double sws = 0.0;
        for (int n2 = 0; n2 < NS; n2++) sws += (DIM == 1) ? ops.wq[n2] : ops.wq[n2 % N] * ops.wq[n2 / N];
        sWsum = sws;
    }
    const int el = tid / NS, nd = tid % NS;
    const int e = blockIdx.x * EPB + el;
    const bool live = e < E;
    // 1. stage combination
    if (live) {
        const double dt = (mode == 0) ? dtp[0] : 0.0;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const size_t g = ((size_t)v * E + e) * NS + nd;
            double val;
            if (mode == 0) {
                const double t = ws[g] + dt * R[g];
                if (stage == 0) val = t;
                else if (stage == 1) val = 0.75 * wn[g] + 0.25 * t;
                else val = (1.0 / 3.0) * wn[g] + (2.0 / 3.0) * t;
            } else {
                val = ws[g];
            }
            sw[el][v][nd] = val;
        }
    }
    __syncthreads();
    // 2. face values (interpolation along the line normal to each face)
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (blockIdx.x * EPB + ell >= E) continue;
        const int f = fp / NFPF, k = fp % NFPF;
        const double* l = (f & 1) ? slp : slm;
        const bool along_x = (DIM == 1) || f < 2;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) s += l[i] * sw[ell][v][(DIM == 1) ? i : (along_x ? k * N + i : i * N + k)];
            sf[ell][v][fp] = s;
        }
    }
    __syncthreads();
    // 3. mean, extrema over V and alpha_i, one thread per (element, component)
    for (int t = tid; t < EPB * NV; t += NT) {
        const int ell = t / NV, v = t % NV;
        const int ee = blockIdx.x * EPB + ell;
        if (ee < E) {
            double s = 0.0;
            for (int n2 = 0; n2 < NS; n2++) s += sW[n2] * sw[ell][v][n2];
            const double mean = s / sWsum;
            long long kmx = dkey(sw[ell][v][0]), kmn = kmx;
            for (int n2 = 1; n2 < NS; n2++) {
                const long long kk = dkey(sw[ell][v][n2]);
                kmx = kk > kmx ? kk : kmx;
                kmn = kk < kmn ? kk : kmn;
            }
            for (int fp = 0; fp < NFP; fp++) {
                const long long kk = dkey(sf[ell][v][fp]);
                kmx = kk > kmx ? kk : kmx;
                kmn = kk < kmn ? kk : kmn;
            }
            const double mx = dunkey(kmx), mn = dunkey(kmn);
            const double lo = bnd[(size_t)v * E + ee];
            const double hi = bnd[((size_t)NV + v) * E + ee];
            const double dmax = mx - mean, dmin = mn - mean;
            double a;
            if (fabs(dmin) < ph.eps || fabs(dmax) < ph.eps) {
                a = ph.eps_rule ? 1.0 : 0.0;
            } else {
                // comparisons written so that a NaN ratio is ignored
                a = 1.0;
                const double t1 = fabs((hi - mean) / dmax);
                const double t2 = fabs((lo - mean) / dmin);
                if (t1 < a) a = t1;
                if (t2 < a) a = t2;
            }
            smean[ell][v] = mean;
            salpha_v[ell][v] = a;
        }
    }
    __syncthreads();
    if (tid < EPB) {
        double a = 1.0;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double b = salpha_v[tid][v];
            if (b < a) a = b;
        }
        salpha[tid] = a;
    }
    __syncthreads();
    // 4. limited state at V.  Pressure floor test without a division first:
    //    P < p_floor  <=>  (gamma-1) (rho E - |m|^2/2) < p_floor rho  (rho > 0);
    //    the margin bounds the rounding of rho E - |m|^2/2 (it can cancel), so the
    //    screen never passes a point the exact test would fail; any element it
    //    flags gets the exact P_min of Eq. 47 below.
    const double gm1 = ph.gamma - 1.0;
    if (live) {
        const double a = salpha[el];
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double m = smean[el][v];
            q[v] = m + a * (sw[el][v][nd] - m);
            sw[el][v][nd] = q[v];
        }
        double mm = q[1] * q[1];
        if (DIM == 2) mm += q[2] * q[2];
        const double X = fma(q[DIM + 1], q[0], -0.5 * mm);
        const double tol = 4e-15 * (fabs(q[DIM + 1] * q[0]) + 0.5 * mm);
        sP[el][nd] = (!(q[0] > 0.0) || gm1 * (X - tol) < ph.p_floor * q[0]) ? -1.0 : 1.0;
    }
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (blockIdx.x * EPB + ell >= E) continue;
        const double a = salpha[ell];
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double m = smean[ell][v];
            q[v] = m + a * (sf[ell][v][fp] - m);
            sf[ell][v][fp] = q[v];
        }
        double mm = q[1] * q[1];
        if (DIM == 2) mm += q[2] * q[2];
        const double X = fma(q[DIM + 1], q[0], -0.5 * mm);
        const double tol = 4e-15 * (fabs(q[DIM + 1] * q[0]) + 0.5 * mm);
        sP[ell][NS + fp] = (!(q[0] > 0.0) || gm1 * (X - tol) < ph.p_floor * q[0]) ? -1.0 : 1.0;
    }
    __syncthreads();
    if (tid < EPB && blockIdx.x * EPB + tid < E) {
        bool low = false;
        for (int n2 = 0; n2 < NS + NFP; n2++) low |= sP[tid][n2] < 0.0;
        double aP = 1.0;
        int taken = 0;
        if (low) {
            // exact P_min over V of the limited state (Eq. 47)
            double pmin = INFINITY, q[NV];
            for (int n2 = 0; n2 < NS + NFP; n2++) {
#pragma unroll
                for (int v = 0; v < NV; v++) q[v] = n2 < NS ? sw[tid][v][n2] : sf[tid][v][n2 - NS];
                const double P = kbl_pressure<DIM>(q, gm1);
                if (P < pmin) pmin = P;
            }
            if (pmin < ph.p_floor) {
#pragma unroll
                for (int v = 0; v < NV; v++) q[v] = smean[tid][v];
                const double Pbar = kbl_pressure<DIM>(q, gm1);
                aP = (Pbar > ph.p_floor) ? fabs((ph.p_floor - Pbar) / (pmin - Pbar)) : 0.0;
                taken = 1;
                atomicAdd(&flags->prelimit, 1ull);
            }
        }
        sPtaken[tid] = taken;
        saP[tid] = aP;
        const int ee = blockIdx.x * EPB + tid;
        if (salpha[tid] < 1.0) atomicAdd(&flags->limited, 1ull);
        if (alpha_out) {
            alpha_out[ee] = salpha[tid];
            alpha_out[E + ee] = aP;
        }
    }
    __syncthreads();
    // 5. write
    if (live) {
        const double aP = saP[el];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double val = sw[el][v][nd];
            if (sPtaken[el]) {
                const double m = smean[el][v];
                val = m + aP * (val - m);
            }
            wout[((size_t)v * E + e) * NS + nd] = val;
        }
    }
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
