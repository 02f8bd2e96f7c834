// kbl_bounds64_body.cuh -- device code of the FP64 kinetic bounds (and helpers the other
// bounds kernels share), used by the FR kernels (kbl_bounds.cu) and by the explicit-stencil
// kernels (kbl_stencil.cu).  See kbl_bounds.cu for the steps and their equations.
#pragma once

#include <cfloat>

#include "kbl_bounds_body.cuh"

namespace kbl_dev {

constexpr int CH = 16;  // states per table chunk

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------
struct StatePrim {
    double U[2];
    double th;     // theta
    double sq;     // sqrt(theta)
    double A;      // rho (2 pi theta)^(-d/2)
    double C;      // theta delta / 2
};

template <int DIM>
__device__ __forceinline__ bool prim_of(const double* q, const Phys& ph, StatePrim& s)
{
    const double rho = q[0];
    const double P = kbl_pressure<DIM>(q, ph.gamma - 1.0);
    if (!(rho > 0.0) || !(P > 0.0)) return false;
    const double th = P / rho;
    s.U[0] = q[1] / rho;
    s.U[1] = (DIM == 2) ? q[2] / rho : 0.0;
    s.th = th;
    s.sq = sqrt(th);
    s.A = (DIM == 1) ? rho / sqrt(2.0 * KBL_PI * th) : rho / (2.0 * KBL_PI * th);
    s.C = 0.5 * (2.0 / (ph.gamma - 1.0) - DIM) * th;
    return true;
}

// Block-wide sum of K doubles per thread; result valid in thread 0.
template <int K, int NT>
__device__ __forceinline__ void block_sum_f64(double (&a)[K], double* sred /* [NT/32][K] */)
{
    constexpr int NW = (NT + 31) / 32;
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (NW > 1) {
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) sred[wid * K + k] = a[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                double s = sred[k];
                for (int q = 1; q < NW; q++) s += sred[q * K + k];
                a[k] = s;
            }
        }
    }
}

// Compensated block-wide sum of K floats per thread (hi + lo pairs);
// result (as doubles) valid in thread 0.
template <int K, int NT>
__device__ __forceinline__ void block_sum_f32c(const float (&a)[K], double (&out)[K], float* sred /* [NW][2K] */)
{
    constexpr int NW = (NT + 31) / 32;
    float hi[K], lo[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        hi[k] = a[k];
        lo[k] = 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi[k], o);
            const float ol = __shfl_xor_sync(0xffffffffu, lo[k], o);
            float s, e;
            two_sum(hi[k], oh, s, e);
            hi[k] = s;
            lo[k] = __fadd_rn(__fadd_rn(lo[k], ol), e);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (NW > 1) {
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                sred[wid * 2 * K + k] = hi[k];
                sred[wid * 2 * K + K + k] = lo[k];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                double s = 0.0;
                for (int q = 0; q < NW; q++) s += (double)sred[q * 2 * K + k] + (double)sred[q * 2 * K + K + k];
                out[k] = s;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; k++) out[k] = (double)hi[k] + (double)lo[k];
    }
}

// Final bounds from the raw sums (see the header comment, step 5-6).
// raw (1D): [Tlo, Thi, nx_hi, nx_lo, px_lo, px_hi, E_lo, E_hi]
// raw (2D): [Tlo, Thi, nx_hi, nx_lo, px_lo, px_hi, ny_hi, ny_lo, py_lo, py_hi, E_lo, E_hi]
template <int DIM>
__device__ __forceinline__ void finalize_bounds(const double* raw, double scale, const Phys& ph,
                                                double* bnd, int E, int e)
{
    constexpr int NV = DIM + 2;
    const double rm = 1.0 - ph.r_fac, rp = 1.0 + ph.r_fac;
    double lo[NV], hi[NV];
    lo[0] = rm * (scale * raw[0]);
    hi[0] = rp * (scale * raw[1]);
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        const double* m = raw + 2 + 4 * d;
        lo[1 + d] = rp * (scale * m[0]) + rm * (scale * m[2]);
        hi[1 + d] = rm * (scale * m[1]) + rp * (scale * m[3]);
    }
    lo[NV - 1] = rm * (scale * raw[2 + 4 * DIM]);
    hi[NV - 1] = rp * (scale * raw[3 + 4 * DIM]);
    if (lo[0] < ph.rho_floor) lo[0] = ph.rho_floor;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        bnd[(size_t)v * E + e] = lo[v];
        bnd[((size_t)NV + v) * E + e] = hi[v];
    }
}

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// 2D, FP64
// ---------------------------------------------------------------------------
template <int NX>
struct B2f64 {
    static constexpr int TX = 2;                 // grid nodes per thread per axis
    static constexpr int TPA = NX / TX;          // threads per axis
    static constexpr int NT = TPA * TPA;
};

// Bounds of element e from a stencil of NST states, FP64, one block of B2f64<NX>::NT threads:
// gather(sS) fills sS[NST][4]; the bounds go to column e of bnd[2][4][E].
template <int NST, int NX, typename Gather>
__device__ __forceinline__ void bounds2d_f64_core(Gather gather, int E, int e, const Phys& ph,
                                                  double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NV = 4;
    constexpr int TX = B2f64<NX>::TX, TPA = B2f64<NX>::TPA, NT = B2f64<NX>::NT;
    constexpr int NW = (NT + 31) / 32;
    __shared__ double sS[NST][NV];
    __shared__ StatePrim sP[NST];
    __shared__ double sEx[CH][NX], sExc[CH][NX], sEy[CH][NX];
    __shared__ double sux[NX], suy[NX], swx[NX], swy[NX];
    __shared__ double sbox[4], sgh[2];
    __shared__ int sbad;
    __shared__ double sred[NW * 12];

    const int tid = threadIdx.x;
    if (tid == 0) sbad = 0;
    gather(sS);
    __syncthreads();
    for (int i = tid; i < NST; i += NT)
        if (!prim_of<2>(sS[i], ph, sP[i])) atomicOr(&sbad, 1);
    __syncthreads();
    if (sbad) {
        if (tid == 0) {
            write_nan(bnd, E, e, NV);
            atomicOr(&flags->nonphysical, 1);
        }
        return;
    }
    if (tid < 4) {
        const int d = tid >> 1, up = tid & 1;
        double b = up ? sP[0].U[d] + ph.k * sP[0].sq : sP[0].U[d] - ph.k * sP[0].sq;
        for (int i = 1; i < NST; i++) {
            const double c = up ? sP[i].U[d] + ph.k * sP[i].sq : sP[i].U[d] - ph.k * sP[i].sq;
            b = up ? fmax(b, c) : fmin(b, c);
        }
        sbox[tid] = b;
    }
    __syncthreads();
    const int nu = ph.nu[0];   // nodes per axis; tile nodes j >= nu sit on the box end with weight 0
    if (tid < 2) sgh[tid] = (sbox[2 * tid + 1] - sbox[2 * tid]) / (nu - 1);
    __syncthreads();
    for (int j = tid; j < 2 * NX; j += NT) {
        const int d = j / NX, jj = j % NX;
        const double lo = sbox[2 * d], h = sgh[d];
        const double u = lo + min(jj, nu - 1) * h;
        const double wq = kbl_qweight(ph, jj, nu) * h;
        if (d == 0) { sux[jj] = u; swx[jj] = wq; }
        else { suy[jj] = u; swy[jj] = wq; }
    }
    const int tx = tid % TPA, ty = tid / TPA;
    unsigned long long tlo[TX][TX], thi[TX][TX], ilo[TX][TX], ihi[TX][TX];
#pragma unroll
    for (int a = 0; a < TX; a++)
#pragma unroll
        for (int b = 0; b < TX; b++) {
            tlo[a][b] = ~0ull; ilo[a][b] = ~0ull;
            thi[a][b] = 0ull; ihi[a][b] = 0ull;
        }
    for (int c0 = 0; c0 < NST; c0 += CH) {
        const int nc = min(CH, NST - c0);
        __syncthreads();
        // row tables by segments of SEG nodes (product recurrence, a few exponentials per segment)
        constexpr int SEG = NX < 16 ? NX : 16, NSG = NX / SEG;
        for (int task = tid; task < nc * 2 * NSG; task += NT) {
            const int i = task / (2 * NSG), axis = (task / NSG) & 1, jb = (task % NSG) * SEG;
            const StatePrim& s = sP[c0 + i];
            if (axis == 0)
                kbl_gauss_segment(s.A, s.U[0], s.th, sbox[0], sgh[0], nu, jb, jb + SEG, [&](int j, double v) {
                    sEx[i][j] = v;
                    sExc[i][j] = s.C * v;
                });
            else
                kbl_gauss_segment(1.0, s.U[1], s.th, sbox[2], sgh[1], nu, jb, jb + SEG,
                                  [&](int j, double v) { sEy[i][j] = v; });
        }
        __syncthreads();
        for (int i = 0; i < nc; i++) {
            double ex[TX], exc[TX], ey[TX];
#pragma unroll
            for (int a = 0; a < TX; a++) {
                ex[a] = sEx[i][tx * TX + a];
                exc[a] = sExc[i][tx * TX + a];
                ey[a] = sEy[i][ty * TX + a];
            }
#pragma unroll
            for (int a = 0; a < TX; a++)
#pragma unroll
                for (int b = 0; b < TX; b++) {
                    const unsigned long long g = __double_as_longlong(ex[a] * ey[b]);
                    const unsigned long long cg = __double_as_longlong(exc[a] * ey[b]);
                    tlo[a][b] = umin64(tlo[a][b], g);
                    thi[a][b] = umax64(thi[a][b], g);
                    ilo[a][b] = umin64(ilo[a][b], cg);
                    ihi[a][b] = umax64(ihi[a][b], cg);
                }
        }
    }
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = 0.0;
#pragma unroll
    for (int a = 0; a < TX; a++)
#pragma unroll
        for (int b = 0; b < TX; b++) {
            const int jx = tx * TX + a, jy = ty * TX + b;
            const double M = swx[jx] * swy[jy];
            const double ux = sux[jx], uy = suy[jy];
            const double Tl = __longlong_as_double(tlo[a][b]), Th = __longlong_as_double(thi[a][b]);
            const double Il = __longlong_as_double(ilo[a][b]), Ih = __longlong_as_double(ihi[a][b]);
            acc[0] += M * Tl;
            acc[1] += M * Th;
            if (ux < 0.0) { acc[2] += M * Th * ux; acc[3] += M * Tl * ux; }
            else { acc[4] += M * Tl * ux; acc[5] += M * Th * ux; }
            if (uy < 0.0) { acc[6] += M * Th * uy; acc[7] += M * Tl * uy; }
            else { acc[8] += M * Tl * uy; acc[9] += M * Th * uy; }
            const double ke = 0.5 * ux * ux + 0.5 * uy * uy;
            acc[10] += M * (Tl * ke + Il);
            acc[11] += M * (Th * ke + Ih);
        }
    block_sum_f64<12, NT>(acc, sred);
    if (tid == 0) finalize_bounds<2>(acc, 1.0, ph, bnd, E, e);
}

}  // namespace kbl_dev
