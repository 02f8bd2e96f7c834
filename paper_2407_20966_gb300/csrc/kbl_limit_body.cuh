// kbl_limit_body.cuh -- device code of the SSP-RK3 stage fused with the
// limiter, shared by the single-mesh kernel (kbl_limit.cu) and the batched
// persistent kernel (kbl_batch.cu).  The steps are listed at the top of
// kbl_limit.cu.
#pragma once

#include "kbl_internal.cuh"

namespace kbl_dev {

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

template <int DIM, int N, int EPB>
struct LimSmem {
    static constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    double sw[EPB][NV][NS];      // state at solution points (then limited)
    double sf[EPB][NV][NFP];     // state at face points (then limited)
    double smean[EPB][NV];
    double salpha_v[EPB][NV];
    double salpha[EPB];
    int slow[EPB];               // some point of V failed the division-free pressure screen
    double saP[EPB];
    int sPtaken[EPB];
    double slm[N], slp[N], sW[NS];
    // exact fast path: per-component box around the mean that holds every value of V
    double sbl[EPB][NV], sbh[EPB][NV];
    double sdmx[EPB][NV], sdmn[EPB][NV];   // node extremes minus the mean
    float sdev[EPB][NV][NS];               // node deviations from the mean (FP32)
    float sfdev[EPB][NV][NFP];             // face-value deviations from the mean (FP32)
    int sfv[EPB][NV], sfast[EPB];

};

// SSP-RK3 stage (mode 0) or limiter only (mode 1, ws = w in place) for elements
// e0 .. e0+min(EPB, nmax)-1 of one mesh, by a block of NT >= EPB*Ns threads.  Starts with a
// barrier so that a block can call it repeatedly.
template <int DIM, int N, int EPB>
__device__ __forceinline__ void stage_limit_block(LimSmem<DIM, N, EPB>& sm, int NT, int mode, int stage,
                                                  const double* wn, const double* ws,
                                                  const double* __restrict__ R,
                                                  const double* __restrict__ bnd, double dt, double* wout,
                                                  double* __restrict__ alpha_out, int E, const FrOps& ops,
                                                  const Phys& ph, DevFlags* flags, int e0, int nmax)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NFPF = (DIM == 1) ? 1 : N;
    auto& sw = sm.sw;
    auto& sf = sm.sf;
    auto& smean = sm.smean;
    auto& salpha_v = sm.salpha_v;
    auto& salpha = sm.salpha;
    auto& slow = sm.slow;
    auto& saP = sm.saP;
    auto& sPtaken = sm.sPtaken;
    auto& slm = sm.slm;
    auto& slp = sm.slp;
    auto& sW = sm.sW;
    auto& sbl = sm.sbl;
    auto& sbh = sm.sbh;
    auto& sfv = sm.sfv;
    auto& sfast = sm.sfast;
    auto& sdmx = sm.sdmx;
    auto& sdmn = sm.sdmn;
    auto& sdev = sm.sdev;
    auto& sfdev = sm.sfdev;
    const int tid = threadIdx.x;
    __syncthreads();   // the block may call this for consecutive element blocks
    if (tid < N) {
        slm[tid] = ops.lm[tid];
        slp[tid] = ops.lp[tid];
    }
    // mean weights, 1 / their sum and Lambda come precomputed with the operators (no FP64
    // arithmetic here: every FP64 instruction holds the slow FP64 pipe however few lanes run)
    if (tid < NS) sW[tid] = (DIM == 1) ? ops.wq[tid] : ops.wm2[tid];
    const double winv = (DIM == 1) ? ops.winv1 : ops.winv2, sLam = ops.lam;
    const int el = tid / NS, nd = tid % NS;
    const int e = e0 + el;
    const bool live = el < EPB && el < nmax && e < E;
    // 1. stage combination
    if (live) {
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
    // 1b. mean and node extrema (FP64), node deviations from the mean (FP64 difference, kept in
    //     FP32), face-value deviations from them in FP32 with a rounding allowance: an exact screen
    //     for alpha = 1.  Every face value lies within its FP32 deviation +- 1e-6 Lambda M of the
    //     mean (M = largest node deviation; Lambda = max sum |l_i(+-1)|), up to the FP64 rounding
    //     of the face interpolation itself, covered by delta.  If both bounds lie beyond all of V
    //     by that margin and the node extremes already clear the epsilon rule, Eq. 37 gives
    //     alpha_i = 1 whatever the exact face values are, so they need not be formed in FP64.
    for (int t = tid; t < EPB * NV; t += NT) {
        const int ell = t / NV, v = t % NV;
        if (e0 + ell >= E || ell >= nmax) continue;
        double sum = 0.0;
        for (int n2 = 0; n2 < NS; n2++) sum += sW[n2] * sw[ell][v][n2];
        const double mean = sum * winv;
        long long kmx = dkey(sw[ell][v][0]), kmn = kmx;
        for (int n2 = 1; n2 < NS; n2++) {
            const long long kk = dkey(sw[ell][v][n2]);
            kmx = kk > kmx ? kk : kmx;
            kmn = kk < kmn ? kk : kmn;
        }
        smean[ell][v] = mean;
        sdmx[ell][v] = dunkey(kmx) - mean;
        sdmn[ell][v] = dunkey(kmn) - mean;
    }
    __syncthreads();
    if (live) {
        // FP32 differences of the truncated values (integer-pipe truncation, one FP32 subtraction):
        // each is within 2^-23 (|w| + |mean|) + 2^-24 |w - mean| of the exact deviation, which
        // the face allowance below covers
#pragma unroll
        for (int v = 0; v < NV; v++) sdev[el][v][nd] = f32_trunc(sw[el][v][nd]) - f32_trunc(smean[el][v]);
    }
    __syncthreads();
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (e0 + ell >= E || ell >= nmax) continue;
        const int f = fp / NFPF, k = fp % NFPF;
        const bool along_x = (DIM == 1) || f < 2;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < N; i++) {
                const float l = (float)((f & 1) ? slp[i] : slm[i]);
                acc = fmaf(l, sdev[ell][v][(DIM == 1) ? i : (along_x ? k * N + i : i * N + k)], acc);
            }
            sfdev[ell][v][fp] = acc;
        }
    }
    __syncthreads();
    for (int t = tid; t < EPB * NV; t += NT) {
        const int ell = t / NV, v = t % NV;
        const int ee = e0 + ell;
        if (ee >= E || ell >= nmax) continue;
        const double mean = smean[ell][v], dmaxn = sdmx[ell][v], dminn = sdmn[ell][v];
        float fmx = -FLT_MAX, fmn = FLT_MAX;
        for (int fp = 0; fp < NFP; fp++) {
            fmx = fmaxf(fmx, sfdev[ell][v][fp]);
            fmn = fminf(fmn, sfdev[ell][v][fp]);
        }
        const double M = fmax(dmaxn, -dminn);
        // FP32 face interpolation (1e-6 of Lambda M) and the truncated node deviations
        // (at most 2^-23 (2 |mean| + M) + 2^-24 M each, below 2.4e-7 (|mean| + M); 5e-7 with margin)
        const double err = sLam * (1e-6 * M + 5e-7 * (fabs(mean) + M)) + 1e-37;
        const double delta = 1e-14 * (fabs(mean) + fmax(fabs(mean + dmaxn), fabs(mean + dminn))) * sLam;
        const double up = fmax(dmaxn, (double)fmx + err) + delta;    // every value of V is below mean + up
        const double dn = fmax(-dminn, -(double)fmn + err) + delta;  // and above mean - dn
        const double lo = bnd[(size_t)v * E + ee];
        const double hi = bnd[((size_t)NV + v) * E + ee];
        sbl[ell][v] = mean - dn;
        sbh[ell][v] = mean + up;
        sfv[ell][v] = (dmaxn >= ph.eps) && (-dminn >= ph.eps) && (hi - mean >= up) && (mean - lo >= dn);
    }
    __syncthreads();
    // 1c. pressure over the box: a lower bound of P on it (rho from its lower end, E from its lower
    //     end, |m|^2 from the larger end of each component) that clears 2 p_floor plus an allowance
    //     for the rounding of the exact pressure test below means no point of V can fail it
    if (tid < EPB) {
        const int ell = tid;
        int fast = 0;
        if (e0 + ell < E && ell < nmax) {
            fast = 1;
#pragma unroll
            for (int v = 0; v < NV; v++) fast &= sfv[ell][v];
            const double rlo = sbl[ell][0];
            double mm = 0.0;
#pragma unroll
            for (int k = 1; k <= DIM; k++) {
                const double a = fmax(fabs(sbl[ell][k]), fabs(sbh[ell][k]));
                mm += a * a;
            }
            const double elo = sbl[ell][DIM + 1];
            const double eabs = fmax(fabs(elo), fabs(sbh[ell][DIM + 1]));
            if (!(rlo > 0.0)) {
                fast = 0;
            } else {
                // (gamma - 1)(elo - mm / (2 rlo)) >= 2 p_floor + 1e-13 (eabs + mm / rlo), multiplied
                // through by rlo > 0: no FP64 division; its few ulp of rounding sit far inside 1e-13
                const double lhs = (ph.gamma - 1.0) * fma(elo, rlo, -0.5 * mm);
                if (!(lhs >= 2.0 * ph.p_floor * rlo + 1e-13 * fma(eabs, rlo, mm))) fast = 0;
            }
        }
        sfast[ell] = fast;
        slow[ell] = 0;
    }
    __syncthreads();
    // 2. face values (interpolation along the line normal to each face)
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (e0 + ell >= E || ell >= nmax || sfast[ell]) continue;
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
        const int ee = e0 + ell;
        if (ee < E && ell < nmax && sfast[ell]) {
            salpha_v[ell][v] = 1.0;
        } else if (ee < E && ell < nmax) {
            const double mean = smean[ell][v];
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
            salpha_v[ell][v] = a;
        }
    }
    __syncthreads();
    if (tid < EPB) {
        // every alpha_i lies in [0, 1] (never NaN: a NaN ratio is not taken), where the order of
        // the bit patterns is the order of the values: the minimum on the integer pipe
        long long ka = __double_as_longlong(1.0);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const long long kb = __double_as_longlong(salpha_v[tid][v]);
            ka = kb < ka ? kb : ka;
        }
        salpha[tid] = __longlong_as_double(ka);
    }
    __syncthreads();
    // 4. limited state at V.  Pressure floor test without a division first:
    //    P < p_floor  <=>  (gamma-1) (rho E - |m|^2/2) < p_floor rho  (rho > 0);
    //    the margin bounds the rounding of rho E - |m|^2/2 (it can cancel), so the
    //    screen never passes a point the exact test would fail; any element it
    //    flags gets the exact P_min of Eq. 47 below.  Elements that passed the exact screen
    //    (alpha = 1 and the box test) keep w~ = w and need no pressure re-limit.
    const double gm1 = ph.gamma - 1.0;
    if (live && !sfast[el]) {
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double a = ph.uncoupled ? salpha_v[el][v] : salpha[el];   // Eq. 38 (or per component)
            const double m = smean[el][v];
            q[v] = m + a * (sw[el][v][nd] - m);
            sw[el][v][nd] = q[v];
        }
        double mm = q[1] * q[1];
        if (DIM == 2) mm += q[2] * q[2];
        const double X = fma(q[DIM + 1], q[0], -0.5 * mm);
        const double tol = 4e-15 * (fabs(q[DIM + 1] * q[0]) + 0.5 * mm);
        if (!(q[0] > 0.0) || gm1 * (X - tol) < ph.p_floor * q[0]) slow[el] = 1;
    }
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (e0 + ell >= E || ell >= nmax || sfast[ell]) continue;
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double a = ph.uncoupled ? salpha_v[ell][v] : salpha[ell];
            const double m = smean[ell][v];
            q[v] = m + a * (sf[ell][v][fp] - m);
            sf[ell][v][fp] = q[v];
        }
        double mm = q[1] * q[1];
        if (DIM == 2) mm += q[2] * q[2];
        const double X = fma(q[DIM + 1], q[0], -0.5 * mm);
        const double tol = 4e-15 * (fabs(q[DIM + 1] * q[0]) + 0.5 * mm);
        if (!(q[0] > 0.0) || gm1 * (X - tol) < ph.p_floor * q[0]) slow[ell] = 1;
    }
    __syncthreads();
    if (tid < EPB && tid < nmax && e0 + tid < E) {
        const bool low = slow[tid] != 0;
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
        const int ee = e0 + tid;
        // alpha in [0, 1]: alpha < 1 on the bit patterns
        if (__double_as_longlong(salpha[tid]) < __double_as_longlong(1.0)) atomicAdd(&flags->limited, 1ull);
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


}  // namespace kbl_dev
