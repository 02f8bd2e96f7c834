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
// so a block builds per-state row tables (Ex, Ey; FP64 kernels also C*Ex) and every
// (state, node) pair then costs two multiplies (g = Ex Ey and C g) and four min/max.
//
// FP64 kernels: the min/max run on the integer pipe as unsigned 64-bit
// compares of the bit patterns (all values are >= +0, where integer order is
// value order), because the GB300 FP64 pipe is ~1/76 of FP32; the row tables
// come from a product recurrence (kbl_gauss_segment), a few exponentials per
// segment of 16 nodes.
// FP32 kernels: FP64 only for X = rho E - |m|^2/2 (rho P / (gamma-1)) with its
// positivity test (and, in 1D, for assembling the final bounds; the 2D kernels
// assemble them in FP32 and widen them exactly); velocities are taken
// relative to the box centre inside the exponentials; pairs of states share
// one packed multiply (__fmul2_rn) and one three-input min/max; the partial
// sums of the threads meet in a pairwise tree (the 1D kernel keeps a
// compensated block sum).
#include <algorithm>
#include <cfloat>

#include "kbl_bounds64_body.cuh"

namespace {

using namespace kbl_dev;

// 4 resident blocks (64 registers): measured 7% faster than the 2 that 128 registers allow
template <int N, int NX>
__global__ void __launch_bounds__(B2f64<NX>::NT, (B2f64<NX>::NT <= 256 ? 4 : 1))
k_bounds2d_f64(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, Phys ph,
               double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NT = B2f64<NX>::NT;
    const int e = blockIdx.x;
    bounds2d_f64_core<N * N + 8 * N, NX>([&](double (*sS)[4]) { gather_states<2, N, NT>(w, wf, m, e, sS); },
                                         m.E, e, ph, bnd, flags);
}

// ---------------------------------------------------------------------------
// 2D, FP32 envelopes and sums (body in kbl_bounds_body.cuh): one block per element
// ---------------------------------------------------------------------------
template <int N, int NX, int TYSEL, bool PAD = false>
__global__ void __launch_bounds__(B2f32<NX, TYSEL>::NT, B2f32<NX, TYSEL>::MINB)
k_bounds2d_f32(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, Phys ph,
               double* __restrict__ bnd, DevFlags* flags)
{
    kbl_grid_dep_sync();
    __shared__ Bounds2dF32Smem<N, NX, TYSEL> sm;
    bounds2d_f32_element<N, NX, TYSEL, PAD>(sm, w, wf, m, blockIdx.x, ph, bnd, flags);
}

// ---------------------------------------------------------------------------
// 1D (FP64 and FP32): one block per element, one thread per velocity node
// (strided), direct evaluation of every Maxwellian.
// ---------------------------------------------------------------------------
constexpr int NT1 = 128;

template <int N, bool F32, bool WIDE = false>
__global__ void __launch_bounds__(NT1)
k_bounds1d(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, Phys ph,
           double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NS = N, NFP = 2, NST = WIDE ? 3 * NS : NS + 2 * NFP, NV = 3;
    constexpr int NW = NT1 / 32;
    __shared__ double sS[NST][NV];
    __shared__ StatePrim sP[NST];
    __shared__ double sbox[2];
    __shared__ int sbad;
    __shared__ double sred[NW * 16];
    const int e = blockIdx.x, tid = threadIdx.x;
    const int NU = ph.nu[0];
    if (tid == 0) sbad = 0;
    if (WIDE) {
        for (int idx = tid; idx < NST * NV; idx += NT1)
            sS[idx / NV][idx % NV] = kbl_wide1d<N>(w, m, e, idx / NV, idx % NV);
    } else {
        gather_states<1, N, NT1>(w, wf, m, e, sS);
    }
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
        const MeshDev m = mesh_of(c);
        if (c->cfg.nu[0] != NX || c->phys.qwf)   // padded tile or weight table: the 4x4 (or narrower) tile
            kbl_launch(k_bounds2d_f32<N, NX, 0, true>, c->E, B2f32<NX, 0>::NT, 0, s, c->pdl, w, wf, m, c->phys, bnd,
                       c->d_flags);
        else if (NX >= 32 && c->bounds_tile == 1)
            kbl_launch(k_bounds2d_f32<N, NX, 2>, c->E, B2f32<NX, 2>::NT, 0, s, c->pdl, w, wf, m, c->phys, bnd,
                       c->d_flags);
        else if (NX >= 32 && c->bounds_tile == 2)
            kbl_launch(k_bounds2d_f32<N, NX, 3>, c->E, B2f32<NX, 3>::NT, 0, s, c->pdl, w, wf, m, c->phys, bnd,
                       c->d_flags);
        else
            kbl_launch(k_bounds2d_f32<N, NX, 0>, c->E, B2f32<NX, 0>::NT, 0, s, c->pdl, w, wf, m, c->phys, bnd,
                       c->d_flags);
    } else
        k_bounds2d_f64<N, NX><<<c->E, B2f64<NX>::NT, 0, s>>>(w, wf, mesh_of(c), c->phys, bnd, c->d_flags);
    return 1;
}

template <int DIM, int N>
int run_bounds(const kbl_ctx* c, const double* w, const double* wf, double* bnd, cudaStream_t s)
{
    if (c->E == 0) return 0;
    if (DIM == 1) {
        const bool f32 = c->cfg.precision == KBL_FP32_MIXED, wide = c->cfg.stencil == 1;
        const MeshDev m = mesh_of(c);
        if (f32 && wide) k_bounds1d<N, true, true><<<c->E, NT1, 0, s>>>(w, wf, m, c->phys, bnd, c->d_flags);
        else if (f32) k_bounds1d<N, true><<<c->E, NT1, 0, s>>>(w, wf, m, c->phys, bnd, c->d_flags);
        else if (wide) k_bounds1d<N, false, true><<<c->E, NT1, 0, s>>>(w, wf, m, c->phys, bnd, c->d_flags);
        else k_bounds1d<N, false><<<c->E, NT1, 0, s>>>(w, wf, m, c->phys, bnd, c->d_flags);
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
