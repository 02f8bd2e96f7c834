// kbl_fr_body.cuh -- device code of the FR residual, shared by the single-mesh
// kernel (kbl_fr.cu) and the batched persistent kernel (kbl_batch.cu).
#pragma once

#include "kbl_internal.cuh"

namespace kbl_dev {

// Storage (FP64) to arithmetic type and back.  For FP32 arithmetic the conversions run on
// the integer pipe (truncation in, exact widening out): a conversion instruction would take
// an FP64-pipe slot, and the FP64 pipe is the slow one.
template <typename T>
__device__ __forceinline__ T from_f64(double x) { return x; }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return f32_trunc(x); }
template <typename T>
__device__ __forceinline__ double to_f64(T x) { return x; }
template <>
__device__ __forceinline__ double to_f64<float>(float x) { return f64_widen(x); }

template <int DIM, int N, typename T, int EPB>
struct RhsSmem {
    static constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    T sF[EPB][DIM][NV][NS];
    T sJ[EPB][NFP][NV];
    T sD[N][N], sgl[N], sgr[N], slm[N], slp[N];
};

// FR residual of elements e0 .. e0+min(EPB, nmax)-1 of one mesh, by a block of NT >= EPB*Ns threads
// (one per solution point; the others only help with the face loop).
//   1. states and physical fluxes at the solution points -> shared memory
//   2. per face point: common flux (Rusanov; HLLC with flux == 1, HLL with flux == 2) of (interior trace,
//      exterior value) minus
//      the interpolated discontinuous flux -> jump J
//   3. per solution point and axis: D F + g_L' J_minus + g_R' J_plus,
//      R = -sum_axes (2 / h_axis) dF/dxi
// T is the arithmetic type; storage is FP64.  Starts with a barrier so that a
// block can call it repeatedly.
template <int DIM, int N, typename T, int EPB>
__device__ __forceinline__ void rhs_block(RhsSmem<DIM, N, T, EPB>& sm, int NT, const double* __restrict__ w,
                                          const double* __restrict__ wf, const MeshDev& m, const FrOps& ops,
                                          double gamma_d, double* __restrict__ R, int e0, int nmax, int flux = 0)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NFPF = (DIM == 1) ? 1 : N;
    auto& sF = sm.sF;
    auto& sJ = sm.sJ;
    auto& sD = sm.sD;
    auto& sgl = sm.sgl;
    auto& sgr = sm.sgr;
    auto& slm = sm.slm;
    auto& slp = sm.slp;
    const int tid = threadIdx.x;
    __syncthreads();
    // FP32: the host-rounded copies (no FP64 conversion instructions here)
    constexpr bool F32 = sizeof(T) == sizeof(float);
    for (int i = tid; i < N * N; i += NT)
        sD[i / N][i % N] = F32 ? (T)ops.Df[i / N][i % N] : (T)ops.D[i / N][i % N];
    if (tid < N) {
        sgl[tid] = F32 ? (T)ops.glf[tid] : (T)ops.gl[tid];
        sgr[tid] = F32 ? (T)ops.grf[tid] : (T)ops.gr[tid];
        slm[tid] = F32 ? (T)ops.lmf[tid] : (T)ops.lm[tid];
        slp[tid] = F32 ? (T)ops.lpf[tid] : (T)ops.lp[tid];
    }
    const int el = tid / NS, nd = tid % NS;
    const int e = e0 + el;
    const bool node_thread = el < EPB && el < nmax && e < m.E;
    const T gamma = from_f64<T>(gamma_d), gm1 = F32 ? gamma - T(1) : from_f64<T>(gamma_d - 1.0);
    // the first face point of this thread: its interior and exterior values are loaded now, so
    // that their latency (the exterior one behind the neighbour index) overlaps step 1
    double pi[NV], pe[NV];
    bool pre = false;
    {
        const int ell = tid / NFP, fp = tid % NFP, ee = e0 + ell;
        if (tid < EPB * NFP && ee < m.E && ell < nmax) {
            pre = true;
#pragma unroll
            for (int v = 0; v < NV; v++) {
                pi[v] = wf[((size_t)v * m.E + ee) * NFP + fp];
                pe[v] = kbl_exterior<DIM, N>(wf, m, ee, fp, v);
            }
        }
    }
    if (node_thread) {
        T q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) q[v] = from_f64<T>(w[((size_t)v * m.E + e) * NS + nd]);
#pragma unroll
        for (int dir = 0; dir < DIM; dir++) {
            T F[NV];
            kbl_flux<DIM, T>(q, dir, gm1, F);
#pragma unroll
            for (int v = 0; v < NV; v++) sF[el][dir][v][nd] = F[v];
        }
    }
    __syncthreads();
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        const int ee = e0 + ell;
        if (ee >= m.E || ell >= nmax) continue;
        const int f = fp / NFPF, k = fp % NFPF, dir = f >> 1, side = f & 1;
        T qi[NV], qe[NV], Fc[NV];
        if (pre && t == tid) {
#pragma unroll
            for (int v = 0; v < NV; v++) {
                qi[v] = from_f64<T>(pi[v]);
                qe[v] = from_f64<T>(pe[v]);
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; v++) {
                qi[v] = from_f64<T>(wf[((size_t)v * m.E + ee) * NFP + fp]);
                qe[v] = from_f64<T>(kbl_exterior<DIM, N>(wf, m, ee, fp, v));
            }
        }
        if (flux == 1) {
            if (side == 0) kbl_hllc<DIM, T>(qe, qi, dir, gamma, Fc);
            else kbl_hllc<DIM, T>(qi, qe, dir, gamma, Fc);
        } else if (flux == 2) {
            if (side == 0) kbl_hll<DIM, T>(qe, qi, dir, gamma, Fc);
            else kbl_hll<DIM, T>(qi, qe, dir, gamma, Fc);
        } else {
            if (side == 0) kbl_rusanov<DIM, T>(qe, qi, dir, gamma, Fc);
            else kbl_rusanov<DIM, T>(qi, qe, dir, gamma, Fc);
        }
        const T* l = side ? slp : slm;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            T FD = T(0);
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int node = (DIM == 1) ? i : (dir == 0 ? k * N + i : i * N + k);
                FD += l[i] * sF[ell][dir][v][node];
            }
            sJ[ell][fp][v] = Fc[v] - FD;
        }
    }
    __syncthreads();
    if (!node_thread) return;
    const int i = (DIM == 1) ? nd : nd % N;
    const int j = (DIM == 1) ? 0 : nd / N;
    const T sx = T(2) / from_f64<T>(m.h[e * DIM + 0]);
    const T sy = (DIM == 2) ? T(2) / from_f64<T>(m.h[e * DIM + 1]) : T(0);
#pragma unroll
    for (int v = 0; v < NV; v++) {
        T dx = T(0);
#pragma unroll
        for (int mm = 0; mm < N; mm++) dx += sD[i][mm] * sF[el][0][v][(DIM == 1) ? mm : j * N + mm];
        dx += sgl[i] * sJ[el][0 * NFPF + j][v] + sgr[i] * sJ[el][1 * NFPF + j][v];
        T r = -sx * dx;
        if (DIM == 2) {
            T dy = T(0);
#pragma unroll
            for (int mm = 0; mm < N; mm++) dy += sD[j][mm] * sF[el][DIM - 1][v][mm * N + i];
            dy += sgl[j] * sJ[el][2 * NFPF + i][v] + sgr[j] * sJ[el][3 * NFPF + i][v];
            r -= sy * dy;
        }
        R[((size_t)v * m.E + e) * NS + nd] = to_f64<T>(r);
    }
}

}  // namespace kbl_dev
