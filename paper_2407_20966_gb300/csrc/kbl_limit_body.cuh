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
    double slm[N], slp[N], sW[NS];
    // FP32 screen (exact for alpha = 1 and the pressure test, see stage_limit_block)
    double sc[EPB][NV];                    // reference value c of each component
    float saf[EPB][NV][NS];                // fl32 of the node values minus c
    float smf[EPB][NV], sem[EPB][NV];      // FP32 mean m' and a bound of |c + m' - mean|
    float sdx[EPB][NV], sdn[EPB][NV];      // largest and smallest node deviation from m'
    float samax[EPB][NV], ssum[EPB][NV];   // max |a_n|, sum W |a_n| / sum W
    float sdev[EPB][NV][NS];               // node deviations from m'
    float sfdev[EPB][NV][NFP];             // face deviations from m' (FP32 interpolation)
    float sbl[EPB][NV], sbh[EPB][NV];      // a box that holds every value of V
    int sfv[EPB][NV], sfast[EPB];
    // the elements the screen did not pass, and those whose pressure re-limit is taken, listed
    // (in any order) so that the exact path's loops run over them alone: FP64 instructions that a
    // warp issues with every lane predicated off still hold the slow FP64 pipe
    int sslow[EPB], staken[EPB], snslow, sntaken;

};

// SSP-RK3 stage (mode 0) or limiter only (mode 1, ws = w in place) for elements
// e0 .. e0+min(EPB, nmax)-1 of one mesh, by a block of NT >= EPB*Ns threads.  Starts with a
// barrier so that a block can call it repeatedly.  STAGE >= 0 fixes the stage (and mode 0) at
// compile time, so that the other stages' combinations are not in the code at all.
template <int DIM, int N, int EPB, bool KEEP = false, int STAGE = -1>
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
    auto& slm = sm.slm;
    auto& slp = sm.slp;
    auto& sW = sm.sW;
    auto& sbl = sm.sbl;
    auto& sbh = sm.sbh;
    auto& sfv = sm.sfv;
    auto& sfast = sm.sfast;
    auto& sc = sm.sc;
    auto& saf = sm.saf;
    auto& smf = sm.smf;
    auto& sem = sm.sem;
    auto& sdx = sm.sdx;
    auto& sdn = sm.sdn;
    auto& samax = sm.samax;
    auto& ssum = sm.ssum;
    auto& sdev = sm.sdev;
    auto& sfdev = sm.sfdev;
    const int tid = threadIdx.x;
    if (STAGE >= 0) {
        mode = 0;
        stage = STAGE;
    }
    __syncthreads();   // the block may call this for consecutive element blocks
    if (tid == 0) {
        sm.snslow = 0;
        sm.sntaken = 0;
    }
    if (tid < N) {
        slm[tid] = ops.lm[tid];
        slp[tid] = ops.lp[tid];
    }
    // mean weights, 1 / their sum and Lambda come precomputed with the operators (no FP64
    // arithmetic here: every FP64 instruction holds the slow FP64 pipe however few lanes run)
    if (tid < NS) sW[tid] = (DIM == 1) ? ops.wq[tid] : ops.wm2[tid];
    const double winv = (DIM == 1) ? ops.winv1 : ops.winv2;
    const int el = tid / NS, nd = tid % NS;
    const int e = e0 + el;
    const bool live = el < EPB && el < nmax && e < E;
    // 1. stage combination; the FP32 screen works on the differences from a reference value c
    //    of each component near the element's values (its node-0 value before the stage)
    if (live) {
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const size_t g = ((size_t)v * E + e) * NS + nd;
            double val;
            if (mode == 0) {
                val = kbl_ssprk3(stage, wn, ws, R, g, dt);
            } else {
                val = ws[g];
            }
            sw[el][v][nd] = val;
            const double c = ws[((size_t)v * E + e) * NS];
            saf[el][v][nd] = f32_trunc(val - c);
            if (nd == 0) sc[el][v] = c;
        }
    }
    __syncthreads();
    // 1b. An exact screen for alpha = 1, in FP32 (GB300 runs FP64 at ~1/76 of the FP32 rate).
    //     Notation per element and component: w_n the FP64 node values, mean = the FP64 mean
    //     the exact path forms, c the reference, a_n = trunc32(fl64(w_n - c)) (|a_n - (w_n - c)|
    //     <= (2^-23 + 2^-53) |w_n - c| + 2^-126), m' = the FP32 weighted mean of the a_n, S' =
    //     the FP32 weighted mean of the |a_n|, A = max |a_n|, C = |c| rounded up to FP32,
    //     d_n = fl32(a_n - m'), M = max |d_n|.  Errors scale with the deviations, except the
    //     FP64 rounding of the exact path itself, which scales with C.
    //   (i)   |c + m' - mean| <= e_m = (NS + 8) 2^-23 S' + (2 NS + 4) 2^-53 (C + S') + tiny: the
    //         FP32 sum (inputs 2^-23, weights 2^-24, NS-term FMA sum NS 2^-24, 1 / sum W and the
    //         product 2 2^-24, relative to S, with a factor 2 to spare) and the FP64 sum and
    //         1 / sum W of the exact mean.
    //   (ii)  each node: |(w_n - mean) - d_n| <= e_node = 2^-23 M + 2^-22 A + e_m + tiny.
    //   (iii) each face value f (FP64 interpolation of the exact path): |(f - mean) - fd| <=
    //         e_face = Lambda (e_node + (N + 3) 2^-24 M) + 1e-13 Lambda (C + A) + tiny, fd the
    //         FP32 interpolation of the d_n (FP32 weights and sum: (N + 2) 2^-24 Lambda M; the
    //         FP64 rounding and sum l_i - 1 of the exact path: below 4 N 2^-53 Lambda (C + A)).
    //   So every value of V minus mean lies in [-dn, up], dn = max(-min d, -min fd) + e_face,
    //   up = max(max d, max fd) + e_face.  The exact path's dmax = fl64(max_V - mean) is then
    //   <= up (1 + 2^-52) and >= max d - e_node; likewise dmin.  Eq. 37 gives alpha_i = 1 when
    //   both clear eps and hi - mean >= up (1 + 2^-52), mean - lo >= dn (1 + 2^-52): checked
    //   below with hb = trunc32(fl64(hi - c)) (2^-22 |hb| + tiny) and m' for mean - c (e_m).
    //   Every FP32 evaluation has at most a few roundings of non-negative terms (2^-24 each),
    //   which the factors (1 + 2^-16) on the right-hand sides and (1 - 2^-20) on the left cover.
    //   Non-finite values: trunc32 maps NaN and |x| >= 2^128 to infinities, which fail
    //   S' <= 1e30 and C <= 1e30; below those bounds every FP32 quantity here stays finite.
    constexpr float TINY = 1e-35f;                  // covers the absolute 2^-126 terms
    constexpr float CM = (float)(NS + 8) * 0x1p-23f;
    constexpr float CM64 = (float)(2 * NS + 4) * 0x1p-53f;
    constexpr float UPF = 1.0f + 0x1p-16f, DNF = 1.0f - 0x1p-20f;
    const float winvf = (DIM == 1) ? ops.winv1f : ops.winv2f;
    for (int t = tid; t < EPB * NV; t += NT) {
        const int ell = t / NV, v = t % NV;
        if (e0 + ell >= E || ell >= nmax) continue;
        float sm_ = 0.0f, sa = 0.0f, amax = -FLT_MAX, amin = FLT_MAX;
#pragma unroll
        for (int n2 = 0; n2 < NS; n2++) {
            const float a = saf[ell][v][n2], wf = (DIM == 1) ? ops.wqf[n2] : ops.wm2f[n2];
            sm_ = fmaf(wf, a, sm_);
            sa = fmaf(wf, fabsf(a), sa);
            amax = fmaxf(amax, a);
            amin = fminf(amin, a);
        }
        const float m = sm_ * winvf;
#pragma unroll
        for (int n2 = 0; n2 < NS; n2++) sdev[ell][v][n2] = saf[ell][v][n2] - m;
        smf[ell][v] = m;
        const float S = sa * winvf;
        const float C = fabsf(f32_trunc(sc[ell][v])) * (1.0f + 0x1p-22f);
        ssum[ell][v] = fmaxf(S, C);
        sem[ell][v] = CM * S + CM64 * (C + S) + TINY;
        sdx[ell][v] = amax - m;   // = max_n d_n: rounding is monotone
        sdn[ell][v] = amin - m;
        samax[ell][v] = fmaxf(amax, -amin);
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
                const float l = (f & 1) ? ops.lpf[i] : ops.lmf[i];
                acc = fmaf(l, sdev[ell][v][(DIM == 1) ? i : (along_x ? k * N + i : i * N + k)], acc);
            }
            sfdev[ell][v][fp] = acc;
        }
    }
    __syncthreads();
    // the bounds are the first input that a programmatic predecessor (the bounds launch) writes:
    // wait for that grid here (a no-op in an ordinary launch)
    kbl_grid_dep_wait();
    for (int t = tid; t < EPB * NV; t += NT) {
        const int ell = t / NV, v = t % NV;
        const int ee = e0 + ell;
        if (ee >= E || ell >= nmax) continue;
        const float m = smf[ell][v], em = sem[ell][v], dx = sdx[ell][v], dnn = sdn[ell][v], A = samax[ell][v];
        float fmx = -FLT_MAX, fmn = FLT_MAX;
        for (int fp = 0; fp < NFP; fp++) {
            fmx = fmaxf(fmx, sfdev[ell][v][fp]);
            fmn = fminf(fmn, sfdev[ell][v][fp]);
        }
        const double c = sc[ell][v];
        const float c32 = f32_trunc(c), C = fabsf(c32) * (1.0f + 0x1p-22f);
        const float lam = ops.lamf;
        const float M = fmaxf(dx, -dnn);
        const float enode = 0x1p-23f * M + 0x1p-22f * A + em + TINY;
        const float eface = lam * (enode + (float)(N + 3) * 0x1p-24f * M) + (1e-13f * lam) * (C + A) + TINY;
        const float up = (fmaxf(dx, fmx) + eface) * UPF;
        const float dn = (fmaxf(-dnn, -fmn) + eface) * UPF;
        const float need = (ph.epsf_up + enode) * UPF;
        const float hb = f32_trunc(bnd[((size_t)NV + v) * E + ee] - c);
        const float lb = f32_trunc(bnd[(size_t)v * E + ee] - c);
        const bool ok = (ssum[ell][v] <= 1e30f) && (dx >= need) && (-dnn >= need) &&
                        ((hb - m) * DNF >= (up + 0x1p-22f * fabsf(hb) + em + TINY) * UPF) &&
                        ((m - lb) * DNF >= (dn + 0x1p-22f * fabsf(lb) + em + TINY) * UPF);
        sfv[ell][v] = ok;
        // every value of V lies in [c + rl, c + rh], rl = m' - dn - e_m, rh = m' + up + e_m; in
        // absolute FP32 terms (c32 = trunc32(c): |c - c32| <= 2^-22 |c32| + tiny, and the
        // rounding of rl, rh and of c32 + r) the box is widened by 2^-22 (|c32 + r| + |c32|) +
        // 2^-23 |r| + tiny
        const float rl = m - (dn + em) * UPF, rh = m + (up + em) * UPF;
        const float bl = c32 + rl, bh = c32 + rh;
        sbl[ell][v] = bl - (0x1p-22f * (fabsf(bl) + fabsf(c32)) + 0x1p-23f * fabsf(rl) + TINY) * UPF;
        sbh[ell][v] = bh + (0x1p-22f * (fabsf(bh) + fabsf(c32)) + 0x1p-23f * fabsf(rh) + TINY) * UPF;
    }
    __syncthreads();
    // 1c. pressure over the box, FP32: with rho >= rlo > 0, E >= elo, |m|^2 <= mm at every point
    //     of V, the exact test below (gamma-1)(X - tol) >= p_floor rho, X = rho E - |m|^2/2, holds
    //     at every point when (gamma-1)(elo rlo - mm/2 - G) >= 2 p_floor rlo: the left side minus
    //     the right grows with rho once it is >= 0 at rlo, and G = 1e-6 (|E|max rlo + mm) covers
    //     the FP32 rounding of elo rlo - mm/2, the exact test's tol (4e-15) and its FP64
    //     rounding; the factor 2 and 1e-36 cover the rounding (or underflow) of p_floor rlo.
    if (tid < EPB) {
        const int ell = tid;
        int fast = 0;
        if (e0 + ell < E && ell < nmax) {
            fast = 1;
#pragma unroll
            for (int v = 0; v < NV; v++) fast &= sfv[ell][v];
            const float rlo = sbl[ell][0];
            float mm = 0.0f;
#pragma unroll
            for (int k = 1; k <= DIM; k++) {
                const float a = fmaxf(fabsf(sbl[ell][k]), fabsf(sbh[ell][k]));
                mm = fmaf(a, a, mm);
            }
            mm *= 1.0f + 0x1p-20f;
            const float elo = sbl[ell][DIM + 1];
            const float eabs = fmaxf(fabsf(elo), fabsf(sbh[ell][DIM + 1]));
            const float Y = fmaf(elo, rlo, -0.5f * mm) - 1e-6f * fmaf(eabs, rlo, mm);
            if (!(rlo > 0.0f) || !(ph.gm1f_down * Y >= 2.0f * ph.pfloorf_up * rlo + 1e-36f)) fast = 0;
            if (!fast) sm.sslow[atomicAdd(&sm.snslow, 1)] = ell;
        }
        sfast[ell] = fast;
        slow[ell] = 0;
    }
    __syncthreads();
    const int nslow = sm.snslow;
    // 2. the exact path, for the elements the screen did not pass: the FP64 mean (the weights
    //    in order, then 1 / sum W) and the face values (interpolation along the line normal to
    //    each face)
    for (int t = tid; t < nslow * NV; t += NT) {
        const int ell = sm.sslow[t / NV], v = t % NV;
        double sum = 0.0;
        for (int n2 = 0; n2 < NS; n2++) sum += sW[n2] * sw[ell][v][n2];
        smean[ell][v] = sum * winv;
    }
    for (int t = tid; t < nslow * NFP; t += NT) {
        const int ell = sm.sslow[t / NFP], fp = t % NFP;
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
        if (e0 + ell < E && ell < nmax && sfast[ell]) salpha_v[ell][v] = 1.0;
    }
    for (int t = tid; t < nslow * NV; t += NT) {
        const int ell = sm.sslow[t / NV], v = t % NV;
        const int ee = e0 + ell;
        {
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
            // counters of the limiter's rarely taken branches (elements the screen passed meet
            // neither: it certifies both deviations above eps and the mean strictly inside)
            if (mean < lo || mean > hi) atomicAdd(&flags->mean_outside, 1ull);
            double a;
            if (fabs(dmin) < ph.eps || fabs(dmax) < ph.eps) {
                atomicAdd(&flags->eps_rule, 1ull);
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
    for (int t = tid; t < nslow * NS; t += NT) {
        const int ell = sm.sslow[t / NS], n2 = t % NS;
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double a = ph.uncoupled ? salpha_v[ell][v] : salpha[ell];   // Eq. 38 (or per component)
            const double m = smean[ell][v];
            q[v] = m + a * (sw[ell][v][n2] - m);
            sw[ell][v][n2] = q[v];
        }
        double mm = q[1] * q[1];
        if (DIM == 2) mm += q[2] * q[2];
        const double X = fma(q[DIM + 1], q[0], -0.5 * mm);
        const double tol = 4e-15 * (fabs(q[DIM + 1] * q[0]) + 0.5 * mm);
        if (!(q[0] > 0.0) || gm1 * (X - tol) < ph.p_floor * q[0]) slow[ell] = 1;
    }
    for (int t = tid; t < nslow * NFP; t += NT) {
        const int ell = sm.sslow[t / NFP], fp = t % NFP;
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
                sm.staken[atomicAdd(&sm.sntaken, 1)] = tid;
                atomicAdd(&flags->prelimit, 1ull);
            }
        }
        saP[tid] = aP;
        const int ee = e0 + tid;
        // alpha in [0, 1]: alpha < 1 on the bit patterns
        if (__double_as_longlong(salpha[tid]) < __double_as_longlong(1.0)) {
            atomicAdd(&flags->limited, 1ull);
            atomicAdd(&flags->alpha_hist[kbl_alpha_bin(salpha[tid])], 1ull);
        }
        if (alpha_out) {
            alpha_out[ee] = salpha[tid];
            alpha_out[E + ee] = aP;
        }
    }
    __syncthreads();
    // 5. the pressure re-limit (Eq. 49) in sw for the elements that take it, then write sw (with
    //    KEEP the written state stays in sw, for a caller that continues with it)
    const int ntaken = sm.sntaken;
    if (ntaken > 0) {   // block-uniform
        for (int t = tid; t < ntaken * NS; t += NT) {
            const int ell = sm.staken[t / NS], n2 = t % NS;
            const double aP = saP[ell];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const double m = smean[ell][v];
                sw[ell][v][n2] = m + aP * (sw[ell][v][n2] - m);
            }
        }
        __syncthreads();
    }
    if (live) {
#pragma unroll
        for (int v = 0; v < NV; v++) wout[((size_t)v * E + e) * NS + nd] = sw[el][v][nd];
    }
}

// Face traces of the state stage_limit_block<..., KEEP = true> just wrote (it is in sw): the
// operations and order of k_traces, so the values equal kbl_traces of that state bit for bit.
template <int DIM, int N, int EPB>
__device__ __forceinline__ void traces_of_block(LimSmem<DIM, N, EPB>& sm, int NT, int E, int e0, int nmax,
                                                double* __restrict__ wf)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NFPF = (DIM == 1) ? 1 : N;
    __syncthreads();
    for (int t = threadIdx.x; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        const int e = e0 + ell;
        if (e >= E || ell >= nmax) continue;
        const int f = fp / NFPF, k = fp % NFPF;
        const bool plus = f & 1;
        const bool along_x = (DIM == 1) || f < 2;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) {
                const double l = plus ? sm.slp[i] : sm.slm[i];
                const int nd = along_x ? k * N + i : i * N + k;
                s += l * sm.sw[ell][v][(DIM == 1) ? i : nd];
            }
            wf[((size_t)v * E + e) * NFP + fp] = s;
        }
    }
}


}  // namespace kbl_dev
