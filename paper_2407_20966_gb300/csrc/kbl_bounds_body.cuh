// kbl_bounds_body.cuh -- device code of the FP32 2D kinetic bounds, shared by
// the single-mesh kernels (kbl_bounds.cu) and the batched persistent kernels
// (kbl_batch.cu).  The method and the precision split are described at the top
// of kbl_bounds.cu.
#pragma once

#include <cfloat>

#include "kbl_internal.cuh"

#ifndef KBL_BOUNDS_MINB
#define KBL_BOUNDS_MINB 10
#endif

namespace kbl_dev {

constexpr float LOG2E = 1.4426950408889634f;

template <int DIM, int N, int NT>
__device__ __forceinline__ void gather_states(const double* __restrict__ w, const double* __restrict__ wf,
                                              const MeshDev& m, int e, double (*sS)[DIM + 2])
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NST = NS + 2 * NFP;
    for (int idx = threadIdx.x; idx < NST * NV; idx += NT) {
        const int v = idx / NST, r = idx % NST;
        double val;
        if (r < NS) val = w[((size_t)v * m.E + e) * NS + r];
        else if (r < NS + NFP) val = wf[((size_t)v * m.E + e) * NFP + (r - NS)];
        else val = kbl_exterior<DIM, N>(wf, m, e, r - NS - NFP, v);
        sS[r][v] = val;
    }
}

// The same copy with one thread per stencil state (2D): the source of a state is found
// once and its four components are loaded together.
template <int N, int NT>
__device__ __forceinline__ void gather_states_by_state(const double* __restrict__ w, const double* __restrict__ wf,
                                                       const MeshDev& m, int e, double (*sS)[4])
{
    constexpr int NS = N * N, NFP = 4 * N, NST = NS + 2 * NFP;
    for (int r = threadIdx.x; r < NST; r += NT) {
        const double* src;
        size_t stride;
        if (r < NS) {
            src = w + (size_t)e * NS + r;
            stride = (size_t)m.E * NS;
        } else if (r < NS + NFP) {
            src = wf + (size_t)e * NFP + (r - NS);
            stride = (size_t)m.E * NFP;
        } else {
            const int fp = r - NS - NFP, f = fp / N, k = fp - f * N;
            const int nb = m.nbr[e * 4 + f];
            if (nb >= 0) {
                src = wf + (size_t)nb * NFP + (f ^ 1) * N + k;
                stride = (size_t)m.E * NFP;
            } else {
                src = m.bc + (size_t)(-nb - 1) * 4;
                stride = 1;
            }
        }
        const double v0 = src[0], v1 = src[stride], v2 = src[2 * stride], v3 = src[3 * stride];
        sS[r][0] = v0;
        sS[r][1] = v1;
        sS[r][2] = v2;
        sS[r][3] = v3;
    }
}

// Error-free transformation: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void write_nan(double* bnd, int E, int e, int nv)
{
    for (int v = 0; v < 2 * nv; v++) bnd[(size_t)v * E + e] = __longlong_as_double(0x7ff8000000000000ll);
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fast_exp2(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}



// ---------------------------------------------------------------------------
// 2D, FP32 envelopes and sums.  FP64 is used only where the path needs it:
// X = rho E - |m|^2 / 2 (= rho P / (gamma - 1), the cancellation-prone,
// positivity-deciding quantity) and its sign test.  Everything else per state
// (U, theta, A, C, the box) and the assembly of the bounds is FP32, because the
// GB300 FP64 pipe runs at ~1/76 of the FP32 rate.
// ---------------------------------------------------------------------------
// Thread tile of the envelope loop: TYSEL 0 = TX x TX with TX = 4 (grids of 32 or more
// points per axis), 2 = 4 x 2, 3 = 2 x 4 (x nodes x y nodes per thread).
template <int NX, int TYSEL = 0>
struct B2f32 {
    static constexpr int TXD = (NX >= 32) ? 4 : (NX >= 16 ? 2 : 1);
    static constexpr bool T24 = TYSEL == 3 && NX >= 32;
    static constexpr int TX = T24 ? 2 : TXD;                                        // x nodes per thread
    static constexpr int TY = T24 ? 4 : ((TYSEL > 0 && TYSEL <= TX) ? TYSEL : TX); // y nodes per thread
    static constexpr int TPX = NX / TX, TPY = NX / TY;
    static constexpr int NT = TPX * TPY;
    static constexpr int MINB = (NT == 64) ? KBL_BOUNDS_MINB : (NT == 128 ? 8 : 1);
    // table position of grid index j: with 4 nodes per thread the two float2
    // halves of a thread's tile are stored NX/2 apart, so the 16-byte loads of
    // the threads of a warp are contiguous (no shared-memory bank conflicts)
    __host__ __device__ static constexpr int pos(int j)
    {
        return TX == 4 ? ((j & 3) >> 1) * (NX / 2) + (j >> 2) * 2 + (j & 1) : j;
    }
    // y tables: same layout when the y tile is 4 wide, natural order otherwise
    __host__ __device__ static constexpr int posy(int j)
    {
        return TY == 4 ? ((j & 3) >> 1) * (NX / 2) + (j >> 2) * 2 + (j & 1) : j;
    }
};

// Warp reduce-scatter of 16 values: afterwards lane L (even) holds the sum over the warp
// of value L / 2.  16 exchanges instead of 16 x 5.  Plain FP32 adds: the 32 partial sums
// meet in a 5-level pairwise tree, whose rounding error is at most 5 ulp of the sum of
// magnitudes (each thread's own 16-term sums add at most 16 more), far inside the 1e-5
// the FP32 bounds are held to.
__device__ __forceinline__ float warp_reduce_scatter16(const float (&v)[16])
{
    const int lane = threadIdx.x & 31;
    float s[8];
    {   // offset 16: keep the upper 8 values on lanes with bit 4 set
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const float keep = up ? v[8 + k] : v[k];
            const float send = up ? v[k] : v[8 + k];
            s[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
#pragma unroll
    for (int step = 0; step < 3; step++) {   // offsets 8, 4, 2
        const int off = 8 >> step;
        const int n = 4 >> step;              // values kept after this step
        const bool up = lane & off;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k >= n) break;
            const float keep = up ? s[n + k] : s[k], send = up ? s[k] : s[n + k];
            s[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return s[0] + __shfl_xor_sync(0xffffffffu, s[0], 1);
}

// Shared memory of one element's FP32 bounds for a stencil of NST_ states.
template <int NST_, int NX, int TYSEL>
struct Bounds2dF32SmemS {
    using SH = B2f32<NX, TYSEL>;
    static constexpr int NST = NST_, NV = 4;
    static constexpr int NSTP = (NST + 1) & ~1;         // padded to pairs (the last state repeated)
    static constexpr int NPAIR = NSTP / 2;
    static constexpr int TX = SH::TX, TY = SH::TY, TPX = SH::TPX, NT = SH::NT;
    static constexpr int NW = (NT + 31) / 32;
    static constexpr int K = 12;
    // The stencil copy and the per-state constants are dead once the row tables are
    // written (a barrier lies between), so they share storage with the tables.
    union __align__(16) {
        struct {
            double sS[NST][NV];
            // per state: velocity, s = sqrt(log2(e) / (2 theta)), A, C
            float sUx[NSTP], sUy[NSTP], sSc[NSTP], sA[NSTP], sC[NSTP];
        } pre;
        struct {
            float2 sEx[NPAIR][NX], sEy[NPAIR][NX];
        } tab;
    } u;
    // per pair of states, for the row tables: (-s Ux', -s Uy') of both states (velocities
    // relative to the box centre), (s, A) of both, C of both
    float4 sPu[NPAIR], sPs[NPAIR];
    float2 sPc[NPAIR];
    float srx[NX], sry[NX];          // grid relative to the box centre
    // per-node moment coefficients, each duplicated into a pair so that one packed FMA updates
    // a (lower, upper) pair of sums: x: q, q u (u<0), q u (u>=0), 1/2 u^2; y: q, q 1/2 u^2,
    // q u (u<0), q u (u>=0)
    float2 sqx[NX], squxn[NX], squxp[NX], skx[NX], sqy[NX], sqky[NX], squyn[NX], squyp[NX];
    float sbox[NW][4];
    int sbad;
    float sred[NW][16];
    float sfin[K];

};

// The FR stencil of an order-N element: N^2 solution points, 4N own and 4N exterior face points.
template <int N, int NX, int TYSEL>
using Bounds2dF32Smem = Bounds2dF32SmemS<N * N + 8 * N, NX, TYSEL>;

// Bounds of one element from a stencil of NST states (one block of SM::NT threads):
// gather(sS) fills sS[NST][4] with the stencil's conservative states; the bounds go to
// column e of bnd[2][4][E].  The block may call it for several elements in a row: it
// starts with a barrier.  PAD: the grid has ph.nu[0] <= NX nodes per axis or a weight table
// (else exactly NX nodes, trapezoidal rule, with the node count and the weights folded
// into the code).
template <int NST_, int NX, int TYSEL, bool PAD, typename Gather>
__device__ __forceinline__ void bounds2d_f32_core(Bounds2dF32SmemS<NST_, NX, TYSEL>& sm, Gather gather, int E, int e,
                                                  const Phys& ph, double* __restrict__ bnd, DevFlags* flags)
{
    using SM = Bounds2dF32SmemS<NST_, NX, TYSEL>;
    using SH = typename SM::SH;
    constexpr int NST = SM::NST, NV = SM::NV, NSTP = SM::NSTP, NPAIR = SM::NPAIR;
    constexpr int TX = SM::TX, TY = SM::TY, TPX = SM::TPX, NT = SM::NT, NW = SM::NW, K = SM::K;
    (void)TY;
    auto& sS = sm.u.pre.sS; auto& sUx = sm.u.pre.sUx; auto& sUy = sm.u.pre.sUy; auto& sSc = sm.u.pre.sSc;
    auto& sA = sm.u.pre.sA; auto& sC = sm.u.pre.sC; auto& sEx = sm.u.tab.sEx;
    auto& sEy = sm.u.tab.sEy; auto& srx = sm.srx;
    auto& sry = sm.sry; auto& sqx = sm.sqx; auto& squxn = sm.squxn; auto& squxp = sm.squxp; auto& skx = sm.skx; auto& sqy = sm.sqy;
    auto& sqky = sm.sqky; auto& squyn = sm.squyn; auto& squyp = sm.squyp; auto& sbox = sm.sbox;
    auto& sbad = sm.sbad; auto& sred = sm.sred; auto& sfin = sm.sfin;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __syncthreads();   // the block may reuse sm for consecutive elements
    if (tid == 0) sbad = 0;
    gather(sS);
    __syncthreads();

    // 1. primitive state of each stencil node, box candidates
    const float gm1 = ph.gm1f, kk = ph.kf, half_delta = ph.half_delta2f;
    float blx = FLT_MAX, bly = FLT_MAX, bhx = -FLT_MAX, bhy = -FLT_MAX;
    int bad = 0;
    for (int i = tid; i < NSTP; i += NT) {
        const double* q = sS[i < NST ? i : NST - 1];
        // rho e rho = rho E - |m|^2 / 2 and the positivity tests in FP64; the FP32 copies by
        // truncation on the integer pipe
        const double X = fma(q[3], q[0], -0.5 * fma(q[2], q[2], q[1] * q[1]));
        if (!kbl_positive(q[0]) || !kbl_positive(X)) bad = 1;
        // reciprocals and the square root by the special-function unit (a few ulp)
        const float r = f32_trunc(q[0]), inv = __fdividef(1.0f, r);
        const float ux = f32_trunc(q[1]) * inv, uy = f32_trunc(q[2]) * inv;
        const float th = gm1 * (f32_trunc(X) * inv) * inv;
        const float rs = rsqrtf(th);              // 1 / sqrt(theta)
        const float sq = th * rs;                 // sqrt(theta)
        sUx[i] = ux;
        sUy[i] = uy;
        sSc[i] = 0.84932180028801904f * rs;       // sqrt(log2(e) / 2) / sqrt(theta)
        sA[i] = r * (0.15915494309189535f * (rs * rs));   // rho / (2 pi theta)
        sC[i] = half_delta * th;
        blx = fminf(blx, ux - kk * sq);
        bhx = fmaxf(bhx, ux + kk * sq);
        bly = fminf(bly, uy - kk * sq);
        bhy = fmaxf(bhy, uy + kk * sq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        blx = fminf(blx, __shfl_xor_sync(0xffffffffu, blx, o));
        bhx = fmaxf(bhx, __shfl_xor_sync(0xffffffffu, bhx, o));
        bly = fminf(bly, __shfl_xor_sync(0xffffffffu, bly, o));
        bhy = fmaxf(bhy, __shfl_xor_sync(0xffffffffu, bhy, o));
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        sbox[wid][0] = blx; sbox[wid][1] = bhx; sbox[wid][2] = bly; sbox[wid][3] = bhy;
        if (bad) atomicOr(&sbad, 1);
    }
    __syncthreads();
    if (sbad) {   // block-uniform
        if (tid == 0) {
            write_nan(bnd, E, e, NV);
            atomicOr(&flags->nonphysical, 1);
        }
        return;
    }
    float lox = sbox[0][0], hix = sbox[0][1], loy = sbox[0][2], hiy = sbox[0][3];
#pragma unroll
    for (int q = 1; q < NW; q++) {
        lox = fminf(lox, sbox[q][0]); hix = fmaxf(hix, sbox[q][1]);
        loy = fminf(loy, sbox[q][2]); hiy = fmaxf(hiy, sbox[q][3]);
    }
    const float cx = 0.5f * (lox + hix), cy = 0.5f * (loy + hiy);
    const int nu = PAD ? ph.nu[0] : NX;   // nodes per axis; tile nodes j >= nu sit on the box end, weight 0
    const float hx = (hix - lox) / (float)(nu - 1), hy = (hiy - loy) / (float)(nu - 1);

    // 2. state velocities and grid relative to the box centre (for the Maxwellians,
    //    which keeps FP32 differences small), absolute grid for the moments
    for (int pr = tid; pr < NPAIR; pr += NT) {
        const float sa = sSc[2 * pr], sb = sSc[2 * pr + 1];
        sm.sPu[pr] = make_float4(-sa * (sUx[2 * pr] - cx), -sb * (sUx[2 * pr + 1] - cx),
                                 -sa * (sUy[2 * pr] - cy), -sb * (sUy[2 * pr + 1] - cy));
        sm.sPs[pr] = make_float4(sa, sb, sA[2 * pr], sA[2 * pr + 1]);
        sm.sPc[pr] = make_float2(sC[2 * pr], sC[2 * pr + 1]);
    }
    for (int j = tid; j < NX; j += NT) {
        const float t = (float)(PAD ? min(j, nu - 1) : j) - 0.5f * (float)(nu - 1);
        const float q = PAD ? kbl_qweight_f(ph, j, nu) : ((j == 0 || j == NX - 1) ? 0.5f : 1.0f);
        const float rx = t * hx, ry = t * hy;
        const float ux = cx + rx, uy = cy + ry;
        srx[j] = rx;
        sry[j] = ry;
        const float qux = q * ux, kx = 0.5f * ux * ux, qky = q * (0.5f * uy * uy);
        const float qxn = qux < 0.0f ? qux : 0.0f, qxp = qux < 0.0f ? 0.0f : qux;
        const float qyn = uy < 0.0f ? q * uy : 0.0f, qyp = uy < 0.0f ? 0.0f : q * uy;
        sqx[j] = make_float2(q, q);
        squxn[j] = make_float2(qxn, qxn);
        squxp[j] = make_float2(qxp, qxp);
        skx[j] = make_float2(kx, kx);
        sqy[j] = make_float2(q, q);
        sqky[j] = make_float2(qky, qky);
        squyn[j] = make_float2(qyn, qyn);
        squyp[j] = make_float2(qyp, qyp);
    }
    __syncthreads();
    // 3. row tables of every state, two states per packed instruction:
    //    Ex = A exp2(-(s (ux - Ux))^2), Ey = exp2(-(s (uy - Uy))^2), s^2 = log2(e) / (2 theta)
    {
        constexpr int ROWS = NT / NX > 0 ? NT / NX : 1;
        const int j = tid % NX;
        const int pj = SH::pos(j), pjy = SH::posy(j);
        const float2 rx = make_float2(srx[j], srx[j]);
        const float2 ry = make_float2(sry[j], sry[j]);
        for (int pr = tid / NX; pr < NPAIR; pr += ROWS) {
            const float4 u = sm.sPu[pr], sa = sm.sPs[pr];
            const float2 s2 = make_float2(sa.x, sa.y);
            const float2 dx = __ffma2_rn(rx, s2, make_float2(u.x, u.y));
            const float2 dy = __ffma2_rn(ry, s2, make_float2(u.z, u.w));
            const float2 ax = __fmul2_rn(dx, dx), ay = __fmul2_rn(dy, dy);
            const float2 ex = __fmul2_rn(make_float2(fast_exp2(-ax.x), fast_exp2(-ax.y)), make_float2(sa.z, sa.w));
            sEx[pr][pj] = ex;
            sEy[pr][pjy] = make_float2(fast_exp2(-ay.x), fast_exp2(-ay.y));
        }
    }
    __syncthreads();
    // 4. envelopes on this thread's TX x TY tile: packed products of a pair of
    //    states, three-input min/max.  The internal-energy weight multiplies the product
    //    (C (Ex Ey)) rather than a C Ex table: the same two products per pair and node, with
    //    one table less to build, store and load (measured 147-149 us against 151 us at 128^2 P3)
    const int tx = tid % TPX, ty = tid / TPX;
    float tlo[TX][TY], thi[TX][TY], ilo[TX][TY], ihi[TX][TY];
#pragma unroll
    for (int a = 0; a < TX; a++)
#pragma unroll
        for (int b = 0; b < TY; b++) {
            tlo[a][b] = FLT_MAX; ilo[a][b] = FLT_MAX;
            thi[a][b] = 0.0f; ihi[a][b] = 0.0f;
        }
    // unroll factor by pair count, measured (fractions of the envelope-pattern peak on the bench
    // workloads): 12 for 24 or 48 pairs (P3 quads: 0.676 against 0.669 at 8), 4 for odd counts
    // (P2 quads, 17 pairs: 0.625 against 0.609 at 8), 8 otherwise (P2 triangles, 12 pairs:
    // 0.574 against 0.553 at 4 and 0.548 at 12); 2 keeps loop and address arithmetic on the ALU
    // pipe the min/max need, and a full unroll overflows the instruction cache
    constexpr int ENV_UNROLL = (NPAIR % 12 == 0 && NPAIR >= 24) ? 12 : (NPAIR % 2 == 1 ? 4 : 8);
#pragma unroll ENV_UNROLL
    for (int pi = 0; pi < NPAIR; pi++) {
        float2 ex[TX], ey[TY];
        const float2 cc = sm.sPc[pi];   // C of both states
#pragma unroll
        for (int a = 0; a < TX; a++) ex[a] = sEx[pi][SH::pos(tx * TX + a)];
#pragma unroll
        for (int b = 0; b < TY; b++) ey[b] = sEy[pi][SH::posy(ty * TY + b)];
#pragma unroll
        for (int a = 0; a < TX; a++)
#pragma unroll
            for (int b = 0; b < TY; b++) {
                const float2 g = __fmul2_rn(ex[a], ey[b]);
                const float2 cg = __fmul2_rn(g, cc);
                tlo[a][b] = fmin3(tlo[a][b], g.x, g.y);
                thi[a][b] = fmax3(thi[a][b], g.x, g.y);
                ilo[a][b] = fmin3(ilo[a][b], cg.x, cg.y);
                ihi[a][b] = fmax3(ihi[a][b], cg.x, cg.y);
            }
    }
    // 5. moments: column sums over this thread's y nodes, then the x weights.
    //    raw = [Tlo, Thi, nx_hi, nx_lo, px_lo, px_hi, ny_hi, ny_lo, py_lo, py_hi, E_lo, E_hi]
    //    (n/p: u < 0 / u >= 0 part of the momentum sums; hx hy and the
    //    relaxation are applied in FP64 at the end)
    //    Every sum pairs with its counterpart of the other envelope, so one packed FMA
    //    updates both; lane by lane the arithmetic and its order are those of scalar FMAs.
    float2 a01 = make_float2(0.f, 0.f), a32 = a01, a45 = a01, a76 = a01, a89 = a01, aE = a01;
#pragma unroll
    for (int a = 0; a < TX; a++) {
        float2 cT = make_float2(0.f, 0.f), cI = cT, cK = cT, cN = cT, cP = cT;
#pragma unroll
        for (int b = 0; b < TY; b++) {
            const int jy = ty * TY + b;
            const float2 T = make_float2(tlo[a][b], thi[a][b]);
            cT = __ffma2_rn(sqy[jy], T, cT);
            cI = __ffma2_rn(sqy[jy], make_float2(ilo[a][b], ihi[a][b]), cI);
            cK = __ffma2_rn(sqky[jy], T, cK);
            cN = __ffma2_rn(squyn[jy], T, cN);
            cP = __ffma2_rn(squyp[jy], T, cP);
        }
        const int jx = tx * TX + a;
        const float2 qx = sqx[jx];
        a01 = __ffma2_rn(qx, cT, a01);
        a32 = __ffma2_rn(squxn[jx], cT, a32);
        a45 = __ffma2_rn(squxp[jx], cT, a45);
        a76 = __ffma2_rn(qx, cN, a76);
        a89 = __ffma2_rn(qx, cP, a89);
        aE = __ffma2_rn(qx, __ffma2_rn(skx[jx], cT, __fadd2_rn(cK, cI)), aE);
    }
    float acc[16];
    acc[0] = a01.x; acc[1] = a01.y;
    acc[2] = a32.y; acc[3] = a32.x;
    acc[4] = a45.x; acc[5] = a45.y;
    acc[6] = a76.y; acc[7] = a76.x;
    acc[8] = a89.x; acc[9] = a89.y;
    acc[10] = aE.x; acc[11] = aE.y;
#pragma unroll
    for (int k = 12; k < 16; k++) acc[k] = 0.0f;
    const float rs = warp_reduce_scatter16(acc);
    if ((lane & 1) == 0 && (lane >> 1) < K) sred[wid][lane >> 1] = rs;
    __syncthreads();
    // 6. assemble the bounds, one raw sum per lane, in FP32 (three more roundings, ~2e-7 of
    //    the bound, next to the ~3e-7 of the sums): an FP64 chain here held the slow FP64 pipe
    //    on every element's critical path.  The FP64 value is the exact widening.
    if (tid < K) {
        float sum = sred[0][tid];
#pragma unroll
        for (int q = 1; q < NW; q++) sum += sred[q][tid];
        // lower-bound terms take (1 - r), upper-bound terms (1 + r)
        const bool upper_env = (tid == 1) || (tid == 2) || (tid == 5) || (tid == 6) || (tid == 9) || (tid == 11);
        sfin[tid] = (upper_env ? ph.rel_hif : ph.rel_lof) * ((hx * hy) * sum);
    }
    __syncthreads();
    if (tid < 2 * NV) {
        const int v = tid % NV, up = tid / NV;
        float valf;
        if (v == 0) valf = up ? sfin[1] : sfin[0];
        else if (v == NV - 1) valf = up ? sfin[11] : sfin[10];
        else {
            const int b0 = 2 + 4 * (v - 1);
            valf = up ? sfin[b0 + 1] + sfin[b0 + 3] : sfin[b0 + 0] + sfin[b0 + 2];
        }
        double val = f64_widen(valf);
        // val >= 0 (a sum of non-negative terms) or NaN: the order of the bit patterns decides
        if (v == 0 && !up && __double_as_longlong(val) < __double_as_longlong(ph.rho_floor)) val = ph.rho_floor;
        bnd[((size_t)up * NV + v) * E + e] = val;
    }
}


// Bounds of element e of an FR mesh (the stencil of Sec. 5: own solution and face points,
// exterior face values).
template <int N, int NX, int TYSEL, bool PAD = false>
__device__ __forceinline__ void bounds2d_f32_element(
    Bounds2dF32Smem<N, NX, TYSEL>& sm, const double* __restrict__ w, const double* __restrict__ wf,
    const MeshDev& m, int e, const Phys& ph, double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NT = B2f32<NX, TYSEL>::NT;
    bounds2d_f32_core<N * N + 8 * N, NX, TYSEL, PAD>(
        sm, [&](double (*sS)[4]) { gather_states_by_state<N, NT>(w, wf, m, e, sS); }, m.E, e, ph, bnd, flags);
}


}  // namespace kbl_dev
