// kbl_bounds.cu -- kinetic bounds of every element (Sec. 3.3-3.8 of the paper).
//
// For element e with stencil S (solution points, own face points, exterior
// face values; Sec. 5):
//   1. primitive state of every node: rho, U = m / rho, theta = P / rho
//      (Eq. 3, Eq. 8); Maxwellian constant A = rho (2 pi theta)^(-d/2);
//      internal-energy weight C = theta delta / 2, delta = 2/(gamma-1) - d
//      (Eq. 44)
//   2. velocity box per axis: [min_S(U - k sqrt(theta)), max_S(U + k sqrt(theta))]
//      (Eq. 45 with the upper end read as U + k sqrt(theta))
//   3. equispaced grid of nu points per axis with trapezoidal weights (Sec. 3.7)
//   4. at every grid node: envelopes Tlo/Thi = min/max_i g_i and Ilo/Ihi =
//      min/max_i C_i g_i (Eq. 32, with separate translational and internal
//      envelopes)
//   5. moments (Eq. 33-36 plus the internal part of the energy, Eq. 42):
//        rho_lo = (1-r) sum M Tlo,                 rho_hi = (1+r) sum M Thi
//        m_lo   = (1+r) sum_{u<0} M Thi u + (1-r) sum_{u>=0} M Tlo u
//        m_hi   = (1-r) sum_{u<0} M Tlo u + (1+r) sum_{u>=0} M Thi u
//        E_lo   = (1-r) sum M (Tlo |u|^2/2 + Ilo),  E_hi likewise with (1+r)
//      where (1 -+ r) is the relaxation of Eq. 40 (it commutes with min/max
//      and the sums, so it is applied once at the end)
//   6. rho_lo <- max(rho_lo, rho_floor) (Sec. 3.8)
//
// 2D kernels use the separable form of the Maxwellian on the tensor grid:
// g_i(ux, uy) = (A_i exp(-(ux-Ux_i)^2/(2 theta_i))) (exp(-(uy-Uy_i)^2/(2 theta_i))),
// so a block builds per-state row tables Ex, C*Ex, Ey and every (state, node)
// pair then costs two multiplies and four min/max.
//
// FP64 kernels: the min/max run on the integer pipe as unsigned 64-bit
// compares of the bit patterns (all values are >= +0, where integer order is
// value order), because the GB300 FP64 pipe is ~1/76 of FP32; the row tables
// come from a product recurrence (kbl_gauss_segment), a few exponentials per
// segment of 16 nodes.
// FP32 kernels: FP64 only for X = rho E - |m|^2/2 (rho P / (gamma-1)) with its
// positivity test and for assembling the final bounds; velocities are taken
// relative to the box centre inside the exponentials; pairs of states share
// one packed multiply (__fmul2_rn) and one three-input min/max; the partial
// sums of the threads meet in a pairwise tree (the 1D kernel keeps a
// compensated block sum).
#include <algorithm>
#include <cfloat>

#include "kbl_bounds_body.cuh"

namespace {

using namespace kbl_dev;

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

// 4 resident blocks (64 registers): measured 7% faster than the 2 that 128 registers allow
template <int N, int NX>
__global__ void __launch_bounds__(B2f64<NX>::NT, 4)
k_bounds2d_f64(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, Phys ph,
               double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NS = N * N, NFP = 4 * N, NST = NS + 2 * NFP, NV = 4;
    constexpr int TX = B2f64<NX>::TX, TPA = B2f64<NX>::TPA, NT = B2f64<NX>::NT;
    constexpr int NW = (NT + 31) / 32;
    __shared__ double sS[NST][NV];
    __shared__ StatePrim sP[NST];
    __shared__ double sEx[CH][NX], sExc[CH][NX], sEy[CH][NX];
    __shared__ double sux[NX], suy[NX], swx[NX], swy[NX];
    __shared__ double sbox[4], sgh[2];
    __shared__ int sbad;
    __shared__ double sred[NW * 12];

    const int e = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) sbad = 0;
    gather_states<2, N, NT>(w, wf, m, e, sS);
    __syncthreads();
    for (int i = tid; i < NST; i += NT)
        if (!prim_of<2>(sS[i], ph, sP[i])) atomicOr(&sbad, 1);
    __syncthreads();
    if (sbad) {
        if (tid == 0) {
            write_nan(bnd, m.E, e, NV);
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
    if (tid == 0) finalize_bounds<2>(acc, 1.0, ph, bnd, m.E, e);
}

// ---------------------------------------------------------------------------
// 2D, FP32 envelopes and sums (body in kbl_bounds_body.cuh): one block per element
// ---------------------------------------------------------------------------
template <int N, int NX, int TYSEL, bool PAD = false>
__global__ void __launch_bounds__(B2f32<NX, TYSEL>::NT, B2f32<NX, TYSEL>::MINB)
k_bounds2d_f32(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, Phys ph,
               double* __restrict__ bnd, DevFlags* flags)
{
    __shared__ Bounds2dF32Smem<N, NX, TYSEL> sm;
    bounds2d_f32_element<N, NX, TYSEL, PAD>(sm, w, wf, m, blockIdx.x, ph, bnd, flags);
}

// ---------------------------------------------------------------------------
// 1D (FP64 and FP32): one block per element, one thread per velocity node
// (strided), direct evaluation of every Maxwellian.
// ---------------------------------------------------------------------------
constexpr int NT1 = 128;

template <int N, bool F32>
__global__ void __launch_bounds__(NT1)
k_bounds1d(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, Phys ph,
           double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NS = N, NFP = 2, NST = NS + 2 * NFP, NV = 3;
    constexpr int NW = NT1 / 32;
    __shared__ double sS[NST][NV];
    __shared__ StatePrim sP[NST];
    __shared__ double sbox[2];
    __shared__ int sbad;
    __shared__ double sred[NW * 16];
    const int e = blockIdx.x, tid = threadIdx.x;
    const int NU = ph.nu[0];
    if (tid == 0) sbad = 0;
    gather_states<1, N, NT1>(w, wf, m, e, sS);
    __syncthreads();
    for (int i = tid; i < NST; i += NT1)
        if (!prim_of<1>(sS[i], ph, sP[i])) atomicOr(&sbad, 1);
    __syncthreads();
    if (sbad) {
        if (tid == 0) {
            write_nan(bnd, m.E, e, NV);
            atomicOr(&flags->nonphysical, 1);
        }
        return;
    }
    if (tid < 2) {
        double b = tid ? sP[0].U[0] + ph.k * sP[0].sq : sP[0].U[0] - ph.k * sP[0].sq;
        for (int i = 1; i < NST; i++) {
            const double c = tid ? sP[i].U[0] + ph.k * sP[i].sq : sP[i].U[0] - ph.k * sP[i].sq;
            b = tid ? fmax(b, c) : fmin(b, c);
        }
        sbox[tid] = b;
    }
    __syncthreads();
    const double lo = sbox[0], h = (sbox[1] - sbox[0]) / (NU - 1);
    if (!F32) {
        double acc[8];
#pragma unroll
        for (int k = 0; k < 8; k++) acc[k] = 0.0;
        for (int j = tid; j < NU; j += NT1) {
            const double u = lo + j * h;
            const double M = kbl_qweight(ph, j, NU) * h;
            double Tl = DBL_MAX, Th = 0.0, Il = DBL_MAX, Ih = 0.0;
#pragma unroll
            for (int i = 0; i < NST; i++) {
                const double d = u - sP[i].U[0];
                const double g = sP[i].A * exp(-(d * d) / (2.0 * sP[i].th));
                const double cg = sP[i].C * g;
                Tl = fmin(Tl, g); Th = fmax(Th, g);
                Il = fmin(Il, cg); Ih = fmax(Ih, cg);
            }
            acc[0] += M * Tl;
            acc[1] += M * Th;
            if (u < 0.0) { acc[2] += M * Th * u; acc[3] += M * Tl * u; }
            else { acc[4] += M * Tl * u; acc[5] += M * Th * u; }
            const double ke = 0.5 * u * u;
            acc[6] += M * (Tl * ke + Il);
            acc[7] += M * (Th * ke + Ih);
        }
        block_sum_f64<8, NT1>(acc, sred);
        if (tid == 0) finalize_bounds<1>(acc, 1.0, ph, bnd, m.E, e);
    } else {
        const double c = 0.5 * (sbox[0] + sbox[1]);
        float Ur[NST], kx[NST], A[NST], C[NST];
#pragma unroll
        for (int i = 0; i < NST; i++) {
            Ur[i] = (float)(sP[i].U[0] - c);
            kx[i] = (float)(1.4426950408889634 / (2.0 * sP[i].th));
            A[i] = (float)sP[i].A;
            C[i] = (float)sP[i].C;
        }
        float acc[8];
#pragma unroll
        for (int k = 0; k < 8; k++) acc[k] = 0.0f;
        for (int j = tid; j < NU; j += NT1) {
            const double ud = lo + j * h;
            const float u = (float)ud, ur = (float)(ud - c);
            const float q = (float)kbl_qweight(ph, j, NU);
            float Tl = FLT_MAX, Th = 0.0f, Il = FLT_MAX, Ih = 0.0f;
#pragma unroll
            for (int i = 0; i < NST; i++) {
                const float d = ur - Ur[i];
                const float g = A[i] * fast_exp2(-(d * d) * kx[i]);
                const float cg = C[i] * g;
                Tl = fminf(Tl, g); Th = fmaxf(Th, g);
                Il = fminf(Il, cg); Ih = fmaxf(Ih, cg);
            }
            Tl *= q; Th *= q; Il *= q; Ih *= q;
            acc[0] += Tl;
            acc[1] += Th;
            if (u < 0.0f) { acc[2] += Th * u; acc[3] += Tl * u; }
            else { acc[4] += Tl * u; acc[5] += Th * u; }
            const float ke = (float)(0.5 * ud * ud);
            acc[6] += Tl * ke + Il;
            acc[7] += Th * ke + Ih;
        }
        double tot[8];
        block_sum_f32c<8, NT1>(acc, tot, reinterpret_cast<float*>(sred));
        if (tid == 0) finalize_bounds<1>(tot, h, ph, bnd, m.E, e);
    }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int N, int NX>
int run2d(const kbl_ctx* c, const double* w, const double* wf, double* bnd, cudaStream_t s)
{
    if (c->cfg.precision == KBL_FP32_MIXED) {
        if (c->cfg.nu[0] != NX || c->phys.qwf)   // padded tile or weight table: the 4x4 (or narrower) tile
            k_bounds2d_f32<N, NX, 0, true><<<c->E, B2f32<NX, 0>::NT, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd,
                                                                            c->d_flags);
        else if (NX >= 32 && c->bounds_tile == 1)
            k_bounds2d_f32<N, NX, 2><<<c->E, B2f32<NX, 2>::NT, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
        else if (NX >= 32 && c->bounds_tile == 2)
            k_bounds2d_f32<N, NX, 3><<<c->E, B2f32<NX, 3>::NT, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
        else
            k_bounds2d_f32<N, NX, 0><<<c->E, B2f32<NX, 0>::NT, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
    } else
        k_bounds2d_f64<N, NX><<<c->E, B2f64<NX>::NT, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
    return 1;
}

template <int DIM, int N>
int run_bounds(const kbl_ctx* c, const double* w, const double* wf, double* bnd, cudaStream_t s)
{
    if (c->E == 0) return 0;
    if (DIM == 1) {
        if (c->cfg.precision == KBL_FP32_MIXED)
            k_bounds1d<N, true><<<c->E, NT1, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
        else
            k_bounds1d<N, false><<<c->E, NT1, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
        return 1;
    }
    switch (kbl_tile_nx(c->cfg.nu[0])) {
        case 8: return run2d<N, 8>(c, w, wf, bnd, s);
        case 16: return run2d<N, 16>(c, w, wf, bnd, s);
        case 32: return run2d<N, 32>(c, w, wf, bnd, s);
        case 64: return run2d<N, 64>(c, w, wf, bnd, s);
    }
    return -1;
}

}  // namespace

int launch_bounds(const kbl_ctx* c, const double* w, const double* wf, double* bnd, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_bounds, c, w, wf, bnd, s);
}
