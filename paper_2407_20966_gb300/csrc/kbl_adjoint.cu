// kbl_adjoint.cu -- hand-written reverse-mode derivatives (vector-Jacobian products) of
// one limited SSP-RK3 step, FP64, two dimensions: face traces, FR residual, kinetic
// bounds, stage update with the limiter, and the entropy functional used as the
// objective.
//
// Non-smooth points take fixed subgradients (the same rule everywhere):
//   * min / max over a set (envelopes of Eq. 32, the box of Eq. 45, extrema over V,
//     P_min of Eq. 47, the Rusanov wavespeed): the first index in the set's order wins
//     ties and receives the whole cotangent;
//   * alpha_i = min(1, ratio_hi, ratio_lo) (Eq. 37): the "1" branch wins ties (zero
//     derivative), then the upper ratio; alpha = min_i alpha_i (Eq. 39): the lowest
//     component wins ties;
//   * the epsilon rule, the density floor of Sec. 3.8, alpha_P = 0 and the sign split of
//     the momentum sums are locally constant: zero derivative.
// Exterior-state cotangents are written into a per-face-point slot that only the
// element across that face writes (wfb_ext), so no atomics are needed.
#include <cfloat>

#include "kbl_adjoint_body.cuh"
#include "kbl_bounds_body.cuh"

namespace {

using namespace kbl_dev;

// ---------------------------------------------------------------------------
// traces: wb[node] += sum over the face points interpolated from it of l * (wfb + wfb_ext)
// ---------------------------------------------------------------------------
template <int N>
__global__ void k_traces_vjp(const double* __restrict__ wfb, const double* __restrict__ wfb_ext,
                             double* __restrict__ wb, int E, FrOps ops)
{
    constexpr int NS = N * N, NFP = 4 * N;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)E * NS) return;
    const int e = (int)(t / NS), nd = (int)(t % NS);
    const int i = nd % N, j = nd / N;
    for (int v = 0; v < 4; v++) {
        const size_t b = ((size_t)v * E + e) * NFP;
        auto g = [&](int fp) { return wfb[b + fp] + (wfb_ext ? wfb_ext[b + fp] : 0.0); };
        const double s = ops.lm[i] * g(0 * N + j) + ops.lp[i] * g(1 * N + j) + ops.lm[j] * g(2 * N + i) +
                         ops.lp[j] * g(3 * N + i);
        wb[((size_t)v * E + e) * NS + nd] += s;
    }
}

// ---------------------------------------------------------------------------
// FR residual (FP64): given Rb, add to wb (solution points), wfb (own face values) and
// wfb_ext (the neighbour's slot for the exterior values).  One block of EPB elements.
// ---------------------------------------------------------------------------
constexpr int EPB_A = 4;

template <int N>
__global__ void __launch_bounds__(EPB_A* N* N)
k_rhs_vjp(const double* __restrict__ w, const double* __restrict__ wf, const double* __restrict__ Rb,
          MeshDev m, FrOps ops, double gamma, double* __restrict__ wb, double* __restrict__ wfb,
          double* __restrict__ wfb_ext)
{
    constexpr int NS = N * N, NFP = 4 * N, NV = 4, NT = EPB_A * NS;
    __shared__ double sRb[EPB_A][NV][NS];
    __shared__ double sFb[EPB_A][2][NV][NS];
    __shared__ double sJb[EPB_A][NFP][NV];
    const int tid = threadIdx.x, el = tid / NS, nd = tid % NS;
    const int e = blockIdx.x * EPB_A + el;
    const bool live = e < m.E;
    const int i = nd % N, j = nd / N;
    if (live)
        for (int v = 0; v < NV; v++) sRb[el][v][nd] = Rb[((size_t)v * m.E + e) * NS + nd];
    __syncthreads();
    double sx = 0.0, sy = 0.0;
    if (live) {
        sx = 2.0 / m.h[e * 2 + 0];
        sy = 2.0 / m.h[e * 2 + 1];
        // volume term: R(i', j) -= sx D[i'][m] F_x(j, m): the flux at node (i, j) collects D[i'][i]
        for (int v = 0; v < NV; v++) {
            double fx = 0.0, fy = 0.0;
            for (int a = 0; a < N; a++) {
                fx += ops.D[a][i] * sRb[el][v][j * N + a];
                fy += ops.D[a][j] * sRb[el][v][a * N + i];
            }
            sFb[el][0][v][nd] = -sx * fx;
            sFb[el][1][v][nd] = -sy * fy;
        }
    }
    __syncthreads();
    // face jumps: J at face 0/1 point k feeds R(i, k) with -sx g_{L,R}'(x_i); faces 2/3 with -sy
    for (int t = tid; t < EPB_A * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP, ee = blockIdx.x * EPB_A + ell;
        if (ee >= m.E) continue;
        const int f = fp / N, k = fp % N, dir = f >> 1, side = f & 1;
        const double s = dir ? 2.0 / m.h[ee * 2 + 1] : 2.0 / m.h[ee * 2 + 0];
        double Jb[NV];
        for (int v = 0; v < NV; v++) {
            double acc = 0.0;
            for (int a = 0; a < N; a++)
                acc += (side ? ops.gr[a] : ops.gl[a]) * sRb[ell][v][dir == 0 ? k * N + a : a * N + k];
            Jb[v] = -s * acc;
            sJb[ell][fp][v] = Jb[v];
        }
        // J = Fc(q_left, q_right) - F^D: the common flux
        double qi[NV], qe[NV], qib[NV] = {0, 0, 0, 0}, qeb[NV] = {0, 0, 0, 0};
        const int nb = m.nbr[ee * 4 + f];
        for (int v = 0; v < NV; v++) {
            qi[v] = wf[((size_t)v * m.E + ee) * NFP + fp];
            qe[v] = nb >= 0 ? wf[((size_t)v * m.E + nb) * NFP + (f ^ 1) * N + k] : m.bc[(-nb - 1) * NV + v];
        }
        if (dir == 0) {
            if (side == 0) rusanov_vjp<2, 0>(qe, qi, gamma, Jb, qeb, qib);
            else rusanov_vjp<2, 0>(qi, qe, gamma, Jb, qib, qeb);
        } else {
            if (side == 0) rusanov_vjp<2, 1>(qe, qi, gamma, Jb, qeb, qib);
            else rusanov_vjp<2, 1>(qi, qe, gamma, Jb, qib, qeb);
        }
        for (int v = 0; v < NV; v++) {
            wfb[((size_t)v * m.E + ee) * NFP + fp] += qib[v];
            if (nb >= 0) wfb_ext[((size_t)v * m.E + nb) * NFP + (f ^ 1) * N + k] += qeb[v];
        }
    }
    __syncthreads();
    if (!live) return;
    // -F^D: the interpolated discontinuous flux at the face points of this node's row / column
    double q[NV], Fxb[NV], Fyb[NV];
    for (int v = 0; v < NV; v++) {
        q[v] = w[((size_t)v * m.E + e) * NS + nd];
        Fxb[v] = sFb[el][0][v][nd] - ops.lm[i] * sJb[el][0 * N + j][v] - ops.lp[i] * sJb[el][1 * N + j][v];
        Fyb[v] = sFb[el][1][v][nd] - ops.lm[j] * sJb[el][2 * N + i][v] - ops.lp[j] * sJb[el][3 * N + i][v];
    }
    double qb[NV] = {0, 0, 0, 0};
    flux_vjp<2, 0>(q, gamma, Fxb, qb);
    flux_vjp<2, 1>(q, gamma, Fyb, qb);
    for (int v = 0; v < NV; v++) wb[((size_t)v * m.E + e) * NS + nd] += qb[v];
}

// ---------------------------------------------------------------------------
// kinetic bounds (FP64, 2D): given bndb = d(objective)/d(bnd), add the cotangents of
// the stencil states to wb (solution points), wfb (own face values) and wfb_ext
// (exterior values, in the slot of the element that owns the trace).
//
// The bounds are B = sum_j M_j c_j(envelopes at u_j, u_j) on the grid u_j of the box
// [lo, hi]; their derivative has three parts:
//   a) through the envelope values: the winning state of each min / max at u_j gets
//      d g_i(u_j) / d(rho_i, U_i, theta_i) times the cotangent of that envelope;
//   b) through the grid: u_j = lo + t_j (hi - lo) and M_j proportional to the box
//      widths, so d B / d lo and d B / d hi collect u-derivatives (of the explicit
//      velocity factors of Eq. 35-36 and 42 and of the winning Maxwellians) and
//      -/+ (bndb . B_j) / (hi - lo);
//   c) the box ends are min / max over the stencil of U -+ k sqrt(theta) (Eq. 45):
//      their cotangents go to the winning states.
// Pass A (per grid point) finds the winners and the envelope cotangents; pass B (per
// stencil state) re-evaluates only the Maxwellians that won and accumulates (a) and
// their share of (b).  The grid is processed in chunks of at most 1024 points.
// ---------------------------------------------------------------------------
constexpr int NT_BV = 256;

struct AdjPrim {
    double rho, U[2], th, sq, A, C;
};

template <int N, int NX>
struct BvShape {
    static constexpr int NS = N * N, NFP = 4 * N, NST = NS + 2 * NFP;
    static constexpr int NPTS = NX * NX, CHUNK = NPTS < 1024 ? NPTS : 1024;
    static constexpr int TPN = NT_BV / NST;  // pass-B threads per stencil state
    // dynamic shared memory: Ex, C Ex, Ey tables, two chunk cotangents, pass-B partials, winners
    static constexpr size_t SMEM = sizeof(double) * (3 * NST * NX + 2 * CHUNK + (size_t)NST * TPN * 4) +
                                   4 * CHUNK;
};

template <int N, int NX>
__global__ void __launch_bounds__(NT_BV)
k_bounds2d_vjp(const double* __restrict__ w, const double* __restrict__ wf, const double* __restrict__ bnd,
               const double* __restrict__ bndb, MeshDev m, Phys ph, double* __restrict__ wb,
               double* __restrict__ wfb, double* __restrict__ wfb_ext, DevFlags* flags)
{
    using SH = BvShape<N, NX>;
    constexpr int NS = SH::NS, NFP = SH::NFP, NST = SH::NST, NV = 4;
    constexpr int CHUNK = SH::CHUNK, TPN = SH::TPN, NT = NT_BV, NW = NT / 32;
    extern __shared__ double dsm[];
    double(*sEx)[NX] = reinterpret_cast<double(*)[NX]>(dsm);
    double(*sExc)[NX] = sEx + NST;
    double(*sEy)[NX] = sExc + NST;
    double* sWTl = dsm + 3 * NST * NX;
    double* sWTh = sWTl + CHUNK;
    double* sacc = sWTh + CHUNK;                                            // [TPN][NST][4]
    unsigned char* sidx = reinterpret_cast<unsigned char*>(sacc + NST * TPN * 4);  // [CHUNK][4]
    __shared__ double sS[NST][NV];
    __shared__ AdjPrim sP[NST];
    __shared__ double snode[NST][4];   // cotangents of (rho at fixed U, theta), U_x, U_y, theta
    __shared__ double sux[NX], suy[NX], swx[NX], swy[NX];
    __shared__ double sbox[4], sbb[4];
    __shared__ double sB[8];
    __shared__ double sred[NW * 4];
    __shared__ int sbad;

    const int e = blockIdx.x, tid = threadIdx.x;
    // an element whose bounds were not used by the limiter (zero cotangent) adds nothing
    double b0 = 0.0;
    if (tid < 8) {
        const int v = tid & 3, up = tid >> 2;
        b0 = bndb[((size_t)up * NV + v) * m.E + e];
        // rho_min = max(raw, rho_floor): the floor branch (ties included) has no derivative
        if (tid == 0 && bnd[e] <= ph.rho_floor) b0 = 0.0;
        sB[tid] = b0;
    }
    if (!__syncthreads_or(b0 != 0.0)) return;
    if (tid == 0) sbad = 0;
    gather_states<2, N, NT>(w, wf, m, e, sS);
    __syncthreads();
    const double gm1 = ph.gamma - 1.0, delta = 2.0 / gm1 - 2.0;
    for (int i = tid; i < NST; i += NT) {
        const double* q = sS[i];
        const double P = kbl_pressure<2>(q, gm1);
        if (!(q[0] > 0.0) || !(P > 0.0)) {
            atomicOr(&sbad, 1);
            continue;
        }
        AdjPrim s;
        s.rho = q[0];
        s.U[0] = q[1] / q[0];
        s.U[1] = q[2] / q[0];
        s.th = P / q[0];
        s.sq = sqrt(s.th);
        s.A = q[0] / (2.0 * KBL_PI * s.th);
        s.C = 0.5 * delta * s.th;
        sP[i] = s;
        snode[i][0] = snode[i][1] = snode[i][2] = snode[i][3] = 0.0;
    }
    __syncthreads();
    if (sbad) {
        if (tid == 0) atomicOr(&flags->nonphysical, 1);
        return;
    }
    // box (Eq. 45): value and, in pass C, the first state attaining it
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
    for (int j = tid; j < 2 * NX; j += NT) {
        const int d = j / NX, jj = j % NX;
        const double lo = sbox[2 * d], hi = sbox[2 * d + 1];
        const double h = (hi - lo) / (NX - 1);
        const double u = lo + jj * h;
        const double wq = (jj == 0 || jj == NX - 1) ? 0.5 * h : h;
        if (d == 0) { sux[jj] = u; swx[jj] = wq; }
        else { suy[jj] = u; swy[jj] = wq; }
    }
    __syncthreads();
    // the same separable tables (and arithmetic) as the forward FP64 kernel, so the
    // winners of every min / max are those of the forward pass
    {
        constexpr int SEG = NX < 16 ? NX : 16, NSG = NX / SEG;
        const double hx = (sbox[1] - sbox[0]) / (NX - 1), hy = (sbox[3] - sbox[2]) / (NX - 1);
        for (int task = tid; task < NST * 2 * NSG; task += NT) {
            const int i = task / (2 * NSG), axis = (task / NSG) & 1, jb = (task % NSG) * SEG;
            const AdjPrim& s = sP[i];
            if (axis == 0)
                kbl_gauss_segment(s.A, s.U[0], s.th, sbox[0], hx, NX, jb, jb + SEG, [&](int j, double v) {
                    sEx[i][j] = v;
                    sExc[i][j] = s.C * v;
                });
            else
                kbl_gauss_segment(1.0, s.U[1], s.th, sbox[2], hy, NX, jb, jb + SEG,
                                  [&](int j, double v) { sEy[i][j] = v; });
        }
    }
    const double rm = 1.0 - ph.r_fac, rp = 1.0 + ph.r_fac;
    const double Lx = sbox[1] - sbox[0], Ly = sbox[3] - sbox[2];
    const double inv_n1 = 1.0 / (NX - 1);
    double bl_x = 0.0, bh_x = 0.0, bl_y = 0.0, bh_y = 0.0;  // box-end cotangents, this thread's share
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c0 = 0; c0 < SH::NPTS; c0 += CHUNK) {
        __syncthreads();
        // pass A: one grid point per thread
        for (int jj = tid; jj < CHUNK; jj += NT) {
            const int j = c0 + jj, jx = j % NX, jy = j / NX;
            const double ux = sux[jx], uy = suy[jy], M = swx[jx] * swy[jy];
            double tl = DBL_MAX, th = -1.0, il = DBL_MAX, ih = -1.0;
            int itl = 0, ith = 0, iil = 0, iih = 0;
            for (int i = 0; i < NST; i++) {
                const double ey = sEy[i][jy];
                const double g = sEx[i][jx] * ey, cg = sExc[i][jx] * ey;
                if (g < tl) { tl = g; itl = i; }
                if (g > th) { th = g; ith = i; }
                if (cg < il) { il = cg; iil = i; }
                if (cg > ih) { ih = cg; iih = i; }
            }
            const double Tl = rm * tl, Th = rp * th, Il = rm * il, Ih = rp * ih;
            const double ke = 0.5 * (ux * ux + uy * uy);
            const double* lb = sB;
            const double* hb = sB + 4;
            // envelope cotangents (relaxed values), Eq. 33-36 and 42 read backwards
            const double cTl = M * (lb[0] + (ux < 0.0 ? hb[1] : lb[1]) * ux + (uy < 0.0 ? hb[2] : lb[2]) * uy + lb[3] * ke);
            const double cTh = M * (hb[0] + (ux < 0.0 ? lb[1] : hb[1]) * ux + (uy < 0.0 ? lb[2] : hb[2]) * uy + hb[3] * ke);
            sWTl[jj] = rm * cTl;
            sWTh[jj] = rp * cTh;
            sidx[jj * 4 + 0] = (unsigned char)itl;
            sidx[jj * 4 + 1] = (unsigned char)ith;
            sidx[jj * 4 + 2] = (unsigned char)iil;
            sidx[jj * 4 + 3] = (unsigned char)iih;
            // explicit velocity factors
            const double TxL = ux < 0.0 ? Th : Tl, TxH = ux < 0.0 ? Tl : Th;
            const double TyL = uy < 0.0 ? Th : Tl, TyH = uy < 0.0 ? Tl : Th;
            const double ubx = M * (TxL * lb[1] + TxH * hb[1] + ux * (Tl * lb[3] + Th * hb[3]));
            const double uby = M * (TyL * lb[2] + TyH * hb[2] + uy * (Tl * lb[3] + Th * hb[3]));
            // bndb . (this point's terms) = M * dB/dM
            const double MM = M * (lb[0] * Tl + hb[0] * Th + (lb[1] * TxL + hb[1] * TxH) * ux +
                                   (lb[2] * TyL + hb[2] * TyH) * uy + lb[3] * (Tl * ke + Il) + hb[3] * (Th * ke + Ih));
            const double tx = jx * inv_n1, ty = jy * inv_n1;
            bl_x += ubx * (1.0 - tx) - MM / Lx;
            bh_x += ubx * tx + MM / Lx;
            bl_y += uby * (1.0 - ty) - MM / Ly;
            bh_y += uby * ty + MM / Ly;
        }
        __syncthreads();
        // pass B: threads (state i, sub) scan the chunk for the points where state i won
        if (tid < NST * TPN) {
            const int i = tid % NST, sub = tid / NST;
            const AdjPrim s = sP[i];
            const double inv_th = 1.0 / s.th;
            for (int jj = sub; jj < CHUNK; jj += TPN) {
                const uchar4 win = reinterpret_cast<const uchar4*>(sidx)[jj];
                const bool wtl = win.x == i, wth = win.y == i, wil = win.z == i, wih = win.w == i;
                if (!(wtl | wth | wil | wih)) continue;
                const int j = c0 + jj, jx = j % NX, jy = j / NX;
                const double ux = sux[jx], uy = suy[jy], M = swx[jx] * swy[jy];
                const double g = sEx[i][jx] * sEy[i][jy];
                const double wI = (wil ? rm * M * sB[3] : 0.0) + (wih ? rp * M * sB[7] : 0.0);
                const double G = (wtl ? sWTl[jj] : 0.0) + (wth ? sWTh[jj] : 0.0) + s.C * wI;
                const double Gg = G * g;
                const double dx = ux - s.U[0], dy = uy - s.U[1];
                acc[0] += Gg / s.rho;
                acc[1] += Gg * dx * inv_th;
                acc[2] += Gg * dy * inv_th;
                acc[3] += Gg * (0.5 * (dx * dx + dy * dy) * inv_th * inv_th - inv_th) + 0.5 * delta * g * wI;
                const double gx = -Gg * dx * inv_th, gy = -Gg * dy * inv_th;
                const double tx = jx * inv_n1, ty = jy * inv_n1;
                bl_x += gx * (1.0 - tx);
                bh_x += gx * tx;
                bl_y += gy * (1.0 - ty);
                bh_y += gy * ty;
            }
        }
    }
    if (tid < NST * TPN) {
        const int i = tid % NST, sub = tid / NST;
#pragma unroll
        for (int k = 0; k < 4; k++) sacc[(sub * NST + i) * 4 + k] = acc[k];
    }
    // box-end cotangents: block sum (fixed order)
    double bb[4] = {bl_x, bh_x, bl_y, bh_y};
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bb[k] += __shfl_xor_sync(0xffffffffu, bb[k], o);
    if ((tid & 31) == 0)
#pragma unroll
        for (int k = 0; k < 4; k++) sred[(tid >> 5) * 4 + k] = bb[k];
    __syncthreads();
    if (tid < 4) {
        double s = 0.0;
        for (int q = 0; q < NW; q++) s += sred[q * 4 + tid];
        sbb[tid] = s;
    }
    for (int i = tid; i < NST; i += NT)
        for (int sub = 0; sub < TPN; sub++)
#pragma unroll
            for (int k = 0; k < 4; k++) snode[i][k] += sacc[(sub * NST + i) * 4 + k];
    __syncthreads();
    // pass C: box ends -> the first state attaining each (ties: lowest stencil index)
    if (tid == 0) {
        for (int c = 0; c < 4; c++) {
            const int d = c >> 1, up = c & 1;
            int best = 0;
            double b = up ? sP[0].U[d] + ph.k * sP[0].sq : sP[0].U[d] - ph.k * sP[0].sq;
            for (int i = 1; i < NST; i++) {
                const double v = up ? sP[i].U[d] + ph.k * sP[i].sq : sP[i].U[d] - ph.k * sP[i].sq;
                if (up ? v > b : v < b) { b = v; best = i; }
            }
            const double cb = sbb[c];
            snode[best][1 + d] += cb;
            snode[best][3] += (up ? 0.5 : -0.5) * ph.k * cb / sP[best].sq;
        }
    }
    __syncthreads();
    // pass D: (rho | U, theta) -> conservative cotangents, scattered to their sources
    for (int i = tid; i < NST; i += NT) {
        const AdjPrim s = sP[i];
        const double rb = snode[i][0], Ub0 = snode[i][1], Ub1 = snode[i][2], tb = snode[i][3];
        const double E = sS[i][3];
        const double qb0 = rb - (Ub0 * s.U[0] + Ub1 * s.U[1]) / s.rho +
                           tb * gm1 * (s.U[0] * s.U[0] + s.U[1] * s.U[1] - E / s.rho) / s.rho;
        const double qb1 = (Ub0 - tb * gm1 * s.U[0]) / s.rho;
        const double qb2 = (Ub1 - tb * gm1 * s.U[1]) / s.rho;
        const double qb3 = tb * gm1 / s.rho;
        const double qb[4] = {qb0, qb1, qb2, qb3};
        if (i < NS) {
            for (int v = 0; v < NV; v++) wb[((size_t)v * m.E + e) * NS + i] += qb[v];
        } else if (i < NS + NFP) {
            for (int v = 0; v < NV; v++) wfb[((size_t)v * m.E + e) * NFP + (i - NS)] += qb[v];
        } else {
            const int fp = i - NS - NFP, f = fp / N, k = fp % N;
            const int nb = m.nbr[e * 4 + f];
            if (nb >= 0)
                for (int v = 0; v < NV; v++) wfb_ext[((size_t)v * m.E + nb) * NFP + (f ^ 1) * N + k] += qb[v];
        }
    }
}

// ---------------------------------------------------------------------------
// SSP-RK3 stage + limiter (FP64, 2D):
//   wo   = a_s wn + b_s (ws + dt R)         (stage combination)
//   out  = mean + aP (w~ - mean),  w~ = mean + alpha (wo - mean)  (Eq. 38, 48)
// Given ob = d(objective)/d(out): wnb (+)= a_s wob, wsb = b_s wob, Rb = b_s dt wob and
// bndb = d(objective)/d(bnd), where wob is the cotangent of wo.  The forward decisions
// (epsilon rule, which ratio of Eq. 37 is smallest, the component giving alpha, the
// point with P_min, whether Eq. 48 is taken) are recomputed from the same inputs with
// the same arithmetic as the forward kernel.
// ---------------------------------------------------------------------------
constexpr int EPB_L = 4;

template <int N>
struct StageVjpSmem {
    static constexpr int NS = N * N, NFP = 4 * N, NV = 4;
    double sw[EPB_L][NV][NS], sf[EPB_L][NV][NFP];      // wo and its face values
    double stb[EPB_L][NV][NS], stfb[EPB_L][NV][NFP];   // cotangents of w~ (nodes, faces)
    double sfb[EPB_L][NV][NFP];                         // cotangents of the face values of wo
    double smean[EPB_L][NV], smb[EPB_L][NV];
    double salpha_v[EPB_L][NV];
    int sbranch[EPB_L][NV], sxarg[EPB_L][NV][2];
    double salpha[EPB_L], saP[EPB_L], sPbar[EPB_L], spmin[EPB_L];
    double sxb[EPB_L][NV];   // cotangent of the extreme point of Eq. 37 of each component
    int staken[EPB_L], sapm[EPB_L], svstar[EPB_L], sxpt[EPB_L][NV];
    double sW[NS];
};

template <int N>
__global__ void __launch_bounds__(EPB_L* N* N)
k_stage_vjp(int stage, double dt, const double* __restrict__ wn, const double* __restrict__ ws,
            const double* __restrict__ R, const double* __restrict__ bnd, const double* __restrict__ ob, int E,
            FrOps ops, Phys ph, int accumulate_wn, double* __restrict__ wnb, double* __restrict__ wsb,
            double* __restrict__ Rb, double* __restrict__ bndb)
{
    constexpr int NS = N * N, NFP = 4 * N, NV = 4, NVP = NS + NFP, NT = EPB_L * NS;
    __shared__ StageVjpSmem<N> sm;
    auto& sw = sm.sw;
    auto& sf = sm.sf;
    auto& stb = sm.stb;
    auto& stfb = sm.stfb;
    auto& sfb = sm.sfb;
    auto& smean = sm.smean;
    auto& smb = sm.smb;
    const double as = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
    const double bs = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
    const int tid = threadIdx.x, el = tid / NS, nd = tid % NS;
    const int e0 = blockIdx.x * EPB_L, e = e0 + el;
    const bool live = e < E;
    const double gm1 = ph.gamma - 1.0;
    // the factor of Eq. 38 that component v of element ell takes (per component if uncoupled)
    auto aeff = [&](int ell, int v) { return ph.uncoupled ? sm.salpha_v[ell][v] : sm.salpha[ell]; };
    if (tid < NS) sm.sW[tid] = ops.wm2[tid];   // the forward kernel's mean: sum W w times 1 / sum W
    // 1. stage combination (the forward kernel's expression)
    if (live)
        for (int v = 0; v < NV; v++) {
            const size_t g = ((size_t)v * E + e) * NS + nd;
            sw[el][v][nd] = kbl_ssprk3(stage, wn, ws, R, g, dt);
        }
    __syncthreads();
    // 2. face values
    for (int t = tid; t < EPB_L * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (e0 + ell >= E) continue;
        const int f = fp / N, k = fp % N;
        const double* l = (f & 1) ? ops.lp : ops.lm;
        for (int v = 0; v < NV; v++) {
            double s = 0.0;
            for (int i = 0; i < N; i++) s += l[i] * sw[ell][v][f < 2 ? k * N + i : i * N + k];
            sf[ell][v][fp] = s;
            stfb[ell][v][fp] = 0.0;
        }
    }
    __syncthreads();
    // 3. mean, extrema over V (first point wins ties), alpha_i and its branch:
    //    0 = constant (epsilon rule, or the 1 of Eq. 37 is smallest), 2 = upper ratio,
    //    3 = lower ratio (ties: 1 before the upper ratio before the lower one)
    for (int t = tid; t < EPB_L * NV; t += NT) {
        const int ell = t / NV, v = t % NV, ee = e0 + ell;
        if (ee >= E) continue;
        double s = 0.0;
        for (int n2 = 0; n2 < NS; n2++) s += sm.sW[n2] * sw[ell][v][n2];
        const double mean = s * ops.winv2;
        double mx = sw[ell][v][0], mn = mx;
        int amx = 0, amn = 0;
        for (int n2 = 1; n2 < NVP; n2++) {
            const double x = n2 < NS ? sw[ell][v][n2] : sf[ell][v][n2 - NS];
            if (x > mx) { mx = x; amx = n2; }
            if (x < mn) { mn = x; amn = n2; }
        }
        const double lo = bnd[(size_t)v * E + ee], hi = bnd[((size_t)NV + v) * E + ee];
        const double dmax = mx - mean, dmin = mn - mean;
        double a;
        int br = 0;
        if (fabs(dmin) < ph.eps || fabs(dmax) < ph.eps) {
            a = ph.eps_rule ? 1.0 : 0.0;
        } else {
            a = 1.0;
            const double t1 = fabs((hi - mean) / dmax);
            const double t2 = fabs((lo - mean) / dmin);
            if (t1 < a) { a = t1; br = 2; }
            if (t2 < a) { a = t2; br = 3; }
        }
        smean[ell][v] = mean;
        smb[ell][v] = 0.0;
        sm.salpha_v[ell][v] = a;
        sm.sbranch[ell][v] = br;
        sm.sxarg[ell][v][0] = amx;
        sm.sxarg[ell][v][1] = amn;
    }
    __syncthreads();
    // 4. alpha (Eq. 39; the lowest component wins ties), P_min over V of w~ (Eq. 47; the
    //    first point wins ties) and the re-limit decision of Eq. 48-49
    if (tid < EPB_L && e0 + tid < E) {
        const int ell = tid;
        double a = 1.0;
        int vs = -1;
        for (int v = 0; v < NV; v++)
            if (sm.salpha_v[ell][v] < a) { a = sm.salpha_v[ell][v]; vs = v; }
        sm.salpha[ell] = a;
        sm.svstar[ell] = vs;
        double pmin = INFINITY, q[NV];
        int apm = 0;
        for (int n2 = 0; n2 < NVP; n2++) {
            for (int v = 0; v < NV; v++) {
                const double mv = smean[ell][v], av = ph.uncoupled ? sm.salpha_v[ell][v] : a;
                q[v] = mv + av * ((n2 < NS ? sw[ell][v][n2] : sf[ell][v][n2 - NS]) - mv);
            }
            const double P = kbl_pressure<2>(q, gm1);
            if (P < pmin) { pmin = P; apm = n2; }
        }
        int taken = 0;
        double aP = 1.0, Pbar = 0.0;
        if (pmin < ph.p_floor) {
            for (int v = 0; v < NV; v++) q[v] = smean[ell][v];
            Pbar = kbl_pressure<2>(q, gm1);
            aP = (Pbar > ph.p_floor) ? fabs((ph.p_floor - Pbar) / (pmin - Pbar)) : 0.0;
            taken = 1;
        }
        sm.staken[ell] = taken;
        sm.saP[ell] = aP;
        sm.sPbar[ell] = Pbar;
        sm.spmin[ell] = pmin;
        sm.sapm[ell] = apm;
    }
    __syncthreads();
    // 5. cotangent of w~ at the nodes through Eq. 48
    if (live)
        for (int v = 0; v < NV; v++) {
            const double o = ob[((size_t)v * E + e) * NS + nd];
            stb[el][v][nd] = sm.staken[el] ? sm.saP[el] * o : o;
        }
    __syncthreads();
    // 6. Eq. 48-49 backwards: the mean's share and aP's cotangent
    if (tid < EPB_L && e0 + tid < E && sm.staken[tid]) {
        const int ell = tid, ee = e0 + ell;
        const double aP = sm.saP[ell];
        double aPb = 0.0;
        for (int v = 0; v < NV; v++) {
            const double mv = smean[ell][v], av = aeff(ell, v);
            double so = 0.0;
            for (int n2 = 0; n2 < NS; n2++) {
                const double o = ob[((size_t)v * E + ee) * NS + n2];
                so += o;
                aPb += o * (av * (sw[ell][v][n2] - mv));
            }
            smb[ell][v] += (1.0 - aP) * so;
        }
        const double Pbar = sm.sPbar[ell], pmin = sm.spmin[ell];
        if (Pbar > ph.p_floor) {
            const double den = pmin - Pbar, rr = (ph.p_floor - Pbar) / den;
            const double sg = rr < 0.0 ? -1.0 : 1.0;
            const double Pbb = sg * aPb * (rr - 1.0) / den;
            const double pmb = -sg * aPb * rr / den;
            double q[NV], qb[NV] = {0, 0, 0, 0};
            for (int v = 0; v < NV; v++) q[v] = smean[ell][v];
            pressure_vjp<2>(q, ph.gamma, Pbb, qb);
            for (int v = 0; v < NV; v++) smb[ell][v] += qb[v];
            const int apm = sm.sapm[ell];
            double qt[NV], qtb[NV] = {0, 0, 0, 0};
            for (int v = 0; v < NV; v++) {
                const double mv = smean[ell][v];
                qt[v] = mv + aeff(ell, v) * ((apm < NS ? sw[ell][v][apm] : sf[ell][v][apm - NS]) - mv);
            }
            pressure_vjp<2>(qt, ph.gamma, pmb, qtb);
            for (int v = 0; v < NV; v++) {
                if (apm < NS) stb[ell][v][apm] += qtb[v];
                else stfb[ell][v][apm - NS] += qtb[v];
            }
        }
    }
    __syncthreads();
    // 7. Eq. 38 backwards: the cotangent of each component's factor (summed into alpha_min's
    //    when coupled), then Eq. 37 through the winning ratio
    if (tid < EPB_L && e0 + tid < E) {
        const int ell = tid, ee = e0 + ell;
        double abv[NV];
        for (int v = 0; v < NV; v++) {
            const double mv = smean[ell][v], av = aeff(ell, v);
            double st = 0.0, ab = 0.0;
            for (int n2 = 0; n2 < NS; n2++) {
                st += stb[ell][v][n2];
                ab += stb[ell][v][n2] * (sw[ell][v][n2] - mv);
            }
            for (int fp = 0; fp < NFP; fp++) {
                st += stfb[ell][v][fp];
                ab += stfb[ell][v][fp] * (sf[ell][v][fp] - mv);
            }
            smb[ell][v] += (1.0 - av) * st;
            abv[v] = ab;
            sm.sxpt[ell][v] = -1;
            sm.sxb[ell][v] = 0.0;
        }
        double bb[2 * NV];
        for (int k = 0; k < 2 * NV; k++) bb[k] = 0.0;
        // the components whose ratio of Eq. 37 carries a derivative, and the cotangent it gets
        for (int v = 0; v < NV; v++) {
            double ab;
            if (ph.uncoupled) {
                ab = abv[v];
            } else {
                if (v != sm.svstar[ell]) continue;
                ab = 0.0;
                for (int u = 0; u < NV; u++) ab += abv[u];
            }
            if (sm.sbranch[ell][v] < 2) continue;
            const int up = sm.sbranch[ell][v] == 2;
            const int xpt = sm.sxarg[ell][v][up ? 0 : 1];
            const double mv = smean[ell][v];
            const double x = xpt < NS ? sw[ell][v][xpt] : sf[ell][v][xpt - NS];
            const double b = up ? bnd[((size_t)NV + v) * E + ee] : bnd[(size_t)v * E + ee];
            const double den = x - mv, rr = (b - mv) / den;
            const double sg = rr < 0.0 ? -1.0 : 1.0;
            bb[(up ? NV : 0) + v] = sg * ab / den;
            sm.sxb[ell][v] = -sg * rr * ab / den;
            sm.sxpt[ell][v] = xpt;
            smb[ell][v] += sg * ab * (rr - 1.0) / den;
        }
        for (int k = 0; k < 2 * NV; k++) bndb[(size_t)k * E + ee] = bb[k];
    }
    __syncthreads();
    // 8. face values of wo: cotangent = alpha * (w~ face cotangent) + the extreme point's share
    for (int t = tid; t < EPB_L * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        if (e0 + ell >= E) continue;
        for (int v = 0; v < NV; v++)
            sfb[ell][v][fp] = aeff(ell, v) * stfb[ell][v][fp] + (sm.sxpt[ell][v] == NS + fp ? sm.sxb[ell][v] : 0.0);
    }
    __syncthreads();
    // 9. nodes: alpha * w~ cotangent + extreme point + mean (weights W / sum W) + faces
    //    (transposed interpolation), then the stage combination backwards
    if (!live) return;
    const int i = nd % N, j = nd / N;
    for (int v = 0; v < NV; v++) {
        double g = aeff(el, v) * stb[el][v][nd] + (sm.sxpt[el][v] == nd ? sm.sxb[el][v] : 0.0);
        g += smb[el][v] * (sm.sW[nd] * ops.winv2);
        g += ops.lm[i] * sfb[el][v][0 * N + j] + ops.lp[i] * sfb[el][v][1 * N + j] +
             ops.lm[j] * sfb[el][v][2 * N + i] + ops.lp[j] * sfb[el][v][3 * N + i];
        const size_t gi = ((size_t)v * E + e) * NS + nd;
        if (accumulate_wn) wnb[gi] += as * g;
        else wnb[gi] = as * g;
        wsb[gi] = bs * g;
        Rb[gi] = bs * dt * g;
    }
}

// ---------------------------------------------------------------------------
// integrated entropy  J = sum_e |J_e| sum_n W_n rho ln(P rho^-gamma), the density-weighted log
// of the physical entropy s = P rho^-gamma of Sec. 6, integrated with the Gauss-Legendre rule,
// and its gradient
// ---------------------------------------------------------------------------
constexpr int NT_ENT = 256;

template <int N>
__global__ void __launch_bounds__(NT_ENT)
k_entropy_partial(const double* __restrict__ w, MeshDev m, FrOps ops, double gamma, double* __restrict__ part)
{
    constexpr int NS = N * N;
    __shared__ double sred[NT_ENT / 32];
    const size_t t = (size_t)blockIdx.x * NT_ENT + threadIdx.x;
    double val = 0.0;
    if (t < (size_t)m.E * NS) {
        const int e = (int)(t / NS), nd = (int)(t % NS);
        double q[4];
        for (int v = 0; v < 4; v++) q[v] = w[((size_t)v * m.E + e) * NS + nd];
        const double P = kbl_pressure<2>(q, gamma - 1.0);
        const double J = 0.25 * m.h[e * 2] * m.h[e * 2 + 1];
        val = J * ops.wq[nd % N] * ops.wq[nd / N] * q[0] * (log(P) - gamma * log(q[0]));
    }
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < NT_ENT / 32; k++) s += sred[k];
        part[blockIdx.x] = s;
    }
}

// fixed-order sum of the per-block partials (one block)
__global__ void __launch_bounds__(NT_ENT) k_sum_partials(const double* __restrict__ part, int n, double* out)
{
    __shared__ double sred[NT_ENT];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += NT_ENT) s += part[k];
    sred[threadIdx.x] = s;
    __syncthreads();
    for (int o = NT_ENT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sred[threadIdx.x] += sred[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sred[0];
}

template <int N>
__global__ void __launch_bounds__(NT_ENT)
k_entropy_vjp(const double* __restrict__ w, MeshDev m, FrOps ops, double gamma, double Jb, double* __restrict__ wb)
{
    // d/dq [rho ln P - gamma rho ln rho] = (rho / P) dP/dq + (ln(P rho^-gamma) - gamma) e_rho
    constexpr int NS = N * N;
    const size_t t = (size_t)blockIdx.x * NT_ENT + threadIdx.x;
    if (t >= (size_t)m.E * NS) return;
    const int e = (int)(t / NS), nd = (int)(t % NS);
    double q[4];
    for (int v = 0; v < 4; v++) q[v] = w[((size_t)v * m.E + e) * NS + nd];
    const double P = kbl_pressure<2>(q, gamma - 1.0);
    const double c = Jb * 0.25 * m.h[e * 2] * m.h[e * 2 + 1] * ops.wq[nd % N] * ops.wq[nd / N];
    double qb[4] = {0, 0, 0, 0};
    pressure_vjp<2>(q, gamma, c * q[0] / P, qb);
    qb[0] += c * (log(P) - gamma * log(q[0]) - gamma);
    for (int v = 0; v < 4; v++) wb[((size_t)v * m.E + e) * NS + nd] = qb[v];
}

// small elementwise helpers
__global__ void k_set_scalar(double* p, double v) { *p = v; }

__global__ void k_add(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}

}  // namespace

// ===========================================================================
// launchers and C ABI
// ===========================================================================
namespace {

kbl_status afail(kbl_ctx* c, kbl_status st, const char* msg)
{
    if (c) c->err = msg;
    return st;
}

kbl_status acheck(kbl_ctx* c, int n, const char* where)
{
    if (n < 0) return afail(c, KBL_EINVAL, "the adjoint needs dim 2 and a compiled order / velocity grid");
    c->launches += n;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
        return KBL_ECUDA;
    }
    return KBL_OK;
}

template <int N>
int run_traces_vjp(const kbl_ctx* c, const double* wfb, const double* wfbx, double* wb, cudaStream_t s)
{
    const size_t total = (size_t)c->E * N * N;
    if (total == 0) return 0;
    k_traces_vjp<N><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(wfb, wfbx, wb, c->E, c->ops);
    return 1;
}

template <int N>
int run_rhs_vjp(const kbl_ctx* c, const double* w, const double* wf, const double* Rb, double* wb, double* wfb,
                double* wfbx, cudaStream_t s)
{
    if (c->E == 0) return 0;
    k_rhs_vjp<N><<<(c->E + EPB_A - 1) / EPB_A, EPB_A * N * N, 0, s>>>(w, wf, Rb, mesh_of(c), c->ops, c->phys.gamma, wb,
                                                                       wfb, wfbx);
    return 1;
}

template <int N, int NX>
int run_bounds_vjp_nx(const kbl_ctx* c, const double* w, const double* wf, const double* bnd, const double* bndb,
                      double* wb, double* wfb, double* wfbx, cudaStream_t s)
{
    const size_t smem = BvShape<N, NX>::SMEM;
    if (cudaFuncSetAttribute(k_bounds2d_vjp<N, NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    k_bounds2d_vjp<N, NX><<<c->E, NT_BV, smem, s>>>(w, wf, bnd, bndb, mesh_of(c), c->phys, wb, wfb, wfbx, c->d_flags);
    return 1;
}

template <int N>
int run_bounds_vjp(const kbl_ctx* c, const double* w, const double* wf, const double* bnd, const double* bndb,
                   double* wb, double* wfb, double* wfbx, cudaStream_t s)
{
    if (c->E == 0) return 0;
    switch (c->cfg.nu[0]) {
        case 8: return run_bounds_vjp_nx<N, 8>(c, w, wf, bnd, bndb, wb, wfb, wfbx, s);
        case 16: return run_bounds_vjp_nx<N, 16>(c, w, wf, bnd, bndb, wb, wfb, wfbx, s);
        case 32: return run_bounds_vjp_nx<N, 32>(c, w, wf, bnd, bndb, wb, wfb, wfbx, s);
        case 64: return run_bounds_vjp_nx<N, 64>(c, w, wf, bnd, bndb, wb, wfb, wfbx, s);
    }
    return -1;
}

template <int N>
int run_stage_vjp(const kbl_ctx* c, int stage, double dt, const double* wn, const double* ws, const double* R,
                  const double* bnd, const double* ob, int acc, double* wnb, double* wsb, double* Rb, double* bndb,
                  cudaStream_t s)
{
    if (c->E == 0) return 0;
    k_stage_vjp<N><<<(c->E + EPB_L - 1) / EPB_L, EPB_L * N * N, 0, s>>>(stage, dt, wn, ws, R, bnd, ob, c->E, c->ops,
                                                                         c->phys, acc, wnb, wsb, Rb, bndb);
    return 1;
}

template <int N>
int run_entropy(const kbl_ctx* c, const double* w, double* part, double* J, cudaStream_t s)
{
    const size_t total = (size_t)c->E * N * N;
    const int nb = (int)((total + NT_ENT - 1) / NT_ENT);
    if (nb > 0) k_entropy_partial<N><<<nb, NT_ENT, 0, s>>>(w, mesh_of(c), c->ops, c->phys.gamma, part);
    k_sum_partials<<<1, NT_ENT, 0, s>>>(part, nb, J);
    return nb > 0 ? 2 : 1;
}

template <int N>
int run_entropy_vjp(const kbl_ctx* c, const double* w, double Jb, double* wb, cudaStream_t s)
{
    const size_t total = (size_t)c->E * N * N;
    if (total == 0) return 0;
    k_entropy_vjp<N><<<(unsigned)((total + NT_ENT - 1) / NT_ENT), NT_ENT, 0, s>>>(w, mesh_of(c), c->ops,
                                                                                   c->phys.gamma, Jb, wb);
    return 1;
}

bool adj_ok(const kbl_ctx* c) { return c && c->mesh_ready && c->cfg.dim == 2; }

// The bounds adjoint differentiates the trapezoidal rule on a full kernel tile.
bool adj_grid_ok(const kbl_ctx* c)
{
    return c->cfg.quadrature == 0 && kbl_tile_nx(c->cfg.nu[0]) == c->cfg.nu[0];
}

// Scratch of the adjoint (grown on demand).  Fixed part: the cotangent buffers of one
// step.  Per step of a segment: its input state, the inputs of stages 1 and 2, and the
// traces, bounds and residual of all three stages, kept by the forward pass of the
// segment so that the reverse pass recomputes nothing.
struct AdjLayout {
    size_t S, F, B;
    size_t fixed() const { return 4 * S + 2 * F + B; }
    size_t per_step() const { return 6 * S + 3 * F + 3 * B + 1; }
    size_t total(int n_steps) const { return fixed() + (size_t)n_steps * per_step(); }
};

AdjLayout adj_layout(const kbl_ctx* c)
{
    AdjLayout l;
    l.S = (size_t)c->nv * c->E * c->ns;
    l.F = (size_t)c->nv * c->E * c->nfp;
    l.B = (size_t)2 * c->nv * c->E;
    return l;
}

kbl_status adj_reserve(kbl_ctx* c, int n_steps)
{
    const size_t need = adj_layout(c).total(n_steps);
    if (c->adj_cap >= need) return KBL_OK;
    cudaStreamSynchronize(c->stream);
    if (c->d_adj) cudaFree(c->d_adj);
    c->d_adj = nullptr;
    c->adj_cap = 0;
    const cudaError_t e = cudaMalloc((void**)&c->d_adj, need * sizeof(double));
    if (e != cudaSuccess) {
        c->d_adj = nullptr;
        c->err = std::string("adjoint scratch: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? KBL_ENOMEM : KBL_ECUDA;
    }
    c->adj_cap = need;
    return KBL_OK;
}

// One SSP-RK3 step with a fixed dt (read from the device scalar dtp), as kbl_step issues it.
// With bnd_keep ([3][2][nv][E]) each stage's bounds are written there instead of the
// context's scratch.
int issue_fixed(kbl_ctx* c, double* w, const double* dtp, double* bnd_keep, cudaStream_t s)
{
    int n = 0, r;
    const double* ws = w;
    double* outs[3] = {c->d_wa, c->d_wb, w};
    const size_t B = (size_t)2 * c->nv * c->E;
    for (int st = 0; st < 3; st++) {
        double* bnd = bnd_keep ? bnd_keep + st * B : c->d_bnd;
        if ((r = launch_traces(c, ws, c->d_wf, s)) < 0) return -1;
        n += r;
        if ((r = launch_bounds(c, ws, c->d_wf, bnd, s)) < 0) return -1;
        n += r;
        if ((r = launch_rhs(c, ws, c->d_wf, c->d_R, s)) < 0) return -1;
        n += r;
        if ((r = launch_stage(c, 0, st, w, ws, c->d_R, bnd, dtp, outs[st], nullptr, s)) < 0) return -1;
        n += r;
        ws = outs[st];
    }
    return n;
}

// The stored forward data of one step.
struct StepStore {
    const double* st[3];   // stage inputs (st[0] = the step's input)
    double* R[3];
    double* wf[3];
    double* bn[3];
    double* dtp;           // device copy of the step's dt
};

StepStore step_store(const kbl_ctx* c, int k, const double* input)
{
    const AdjLayout L = adj_layout(c);
    double* p = c->d_adj + L.fixed() + (size_t)k * L.per_step();
    StepStore S;
    S.st[0] = input;
    S.st[1] = p + L.S;
    S.st[2] = p + 2 * L.S;
    p += 3 * L.S;
    for (int i = 0; i < 3; i++) S.R[i] = p + i * L.S;
    p += 3 * L.S;
    for (int i = 0; i < 3; i++) S.wf[i] = p + i * L.F;
    p += 3 * L.F;
    for (int i = 0; i < 3; i++) S.bn[i] = p + i * L.B;
    p += 3 * L.B;
    S.dtp = p;
    return S;
}

// Input-state slot of step k of a segment (k >= 1).
double* step_input_slot(const kbl_ctx* c, int k)
{
    const AdjLayout L = adj_layout(c);
    return c->d_adj + L.fixed() + (size_t)k * L.per_step();
}

// Forward of one step keeping every stage's traces, bounds and residual; the step's
// output goes to `out` (skipped when out is null).
int issue_step_store(kbl_ctx* c, const StepStore& S, double dt, double* out, bool have_bounds, cudaStream_t s)
{
    int n = 1, r;
    k_set_scalar<<<1, 1, 0, s>>>(S.dtp, dt);
    for (int k = 0; k < 3; k++) {
        if ((r = launch_traces(c, S.st[k], S.wf[k], s)) < 0) return -1;
        n += r;
        if (!have_bounds) {
            if ((r = launch_bounds(c, S.st[k], S.wf[k], S.bn[k], s)) < 0) return -1;
            n += r;
        }
        if ((r = launch_rhs(c, S.st[k], S.wf[k], S.R[k], s)) < 0) return -1;
        n += r;
        double* o = k < 2 ? const_cast<double*>(S.st[k + 1]) : out;
        if (o) {
            if ((r = launch_stage(c, 0, k, S.st[0], S.st[k], S.R[k], S.bn[k], S.dtp, o, nullptr, s)) < 0) return -1;
            n += r;
        }
    }
    return n;
}

template <int N>
int reverse_stages(kbl_ctx* c, const StepStore& S, double dt, double* wbar, cudaStream_t s)
{
    const AdjLayout L = adj_layout(c);
    double* p = c->d_adj;
    double* wnb = p;
    double* wsb[2] = {p + L.S, p + 2 * L.S};
    double* Rb = p + 3 * L.S;
    double* wfb = p + 4 * L.S;
    double* wfbx = wfb + L.F;
    double* bndb = wfb + 2 * L.F;
    int n = 0;
    const double* ob = wbar;
    for (int k = 2; k >= 0; k--) {
        double* sb = wsb[k & 1];
        n += run_stage_vjp<N>(c, k, dt, S.st[0], S.st[k], S.R[k], S.bn[k], ob, k != 2, wnb, sb, Rb, bndb, s);
        cudaMemsetAsync(wfb, 0, 2 * L.F * sizeof(double), s);
        n += run_rhs_vjp<N>(c, S.st[k], S.wf[k], Rb, sb, wfb, wfbx, s);
        const int r = run_bounds_vjp<N>(c, S.st[k], S.wf[k], S.bn[k], bndb, sb, wfb, wfbx, s);
        if (r < 0) return -1;
        n += r;
        n += run_traces_vjp<N>(c, wfb, wfbx, sb, s);
        ob = sb;
    }
    // stage 0's input is the step's input itself: its cotangent adds to the wn part
    k_add<<<(unsigned)((L.S + 255) / 256), 256, 0, s>>>(wnb, ob, wbar, L.S);
    return n + 1;
}

// Reverse of one step from its stored forward data: wbar (cotangent of the step's
// output) is replaced by the cotangent of its input.
int issue_step_reverse(kbl_ctx* c, const StepStore& S, double dt, double* wbar, cudaStream_t s)
{
    switch (c->ops.n) {
        case 2: return reverse_stages<2>(c, S, dt, wbar, s);
        case 3: return reverse_stages<3>(c, S, dt, wbar, s);
        case 4: return reverse_stages<4>(c, S, dt, wbar, s);
        case 5: return reverse_stages<5>(c, S, dt, wbar, s);
        case 6: return reverse_stages<6>(c, S, dt, wbar, s);
    }
    return -1;
}

// Stage bounds of step k from a caller's array [n][3][2][nv][E] when given.
StepStore with_bounds(const kbl_ctx* c, StepStore S, const double* bnd_in, int k)
{
    if (bnd_in) {
        const size_t B = adj_layout(c).B;
        for (int i = 0; i < 3; i++) S.bn[i] = const_cast<double*>(bnd_in) + ((size_t)k * 3 + i) * B;
    }
    return S;
}

// n fixed-dt steps from w0 backwards: forward keeping everything (the stage bounds come
// from bnd_in when given), then the reverse.
int issue_segment(kbl_ctx* c, const double* w0, const double* dts, int n, const double* bnd_in, double* wbar,
                  cudaStream_t s)
{
    int launches = 0;
    for (int k = 0; k < n; k++) {
        const StepStore S = with_bounds(c, step_store(c, k, k == 0 ? w0 : step_input_slot(c, k)), bnd_in, k);
        const int r = issue_step_store(c, S, dts[k], k + 1 < n ? step_input_slot(c, k + 1) : nullptr,
                                       bnd_in != nullptr, s);
        if (r < 0) return -1;
        launches += r;
    }
    for (int k = n - 1; k >= 0; k--) {
        const StepStore S = with_bounds(c, step_store(c, k, k == 0 ? w0 : step_input_slot(c, k)), bnd_in, k);
        const int r = issue_step_reverse(c, S, dts[k], wbar, s);
        if (r < 0) return -1;
        launches += r;
    }
    return launches;
}

}  // namespace

void kbl_adjoint_release(kbl_ctx* c)
{
    if (c->d_adj) cudaFree(c->d_adj);
    c->d_adj = nullptr;
    c->adj_cap = 0;
    if (c->d_ent) cudaFree(c->d_ent);
    c->d_ent = nullptr;
    c->ent_cap = 0;
}

extern "C" {

kbl_status kbl_traces_vjp(kbl_ctx* c, const double* wfb, const double* wfb_ext, double* wb)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (c->E > 0 && (!wfb || !wb)) return afail(c, KBL_EINVAL, "null array");
    int r = -1;
    switch (c->ops.n) {
        case 2: r = run_traces_vjp<2>(c, wfb, wfb_ext, wb, c->stream); break;
        case 3: r = run_traces_vjp<3>(c, wfb, wfb_ext, wb, c->stream); break;
        case 4: r = run_traces_vjp<4>(c, wfb, wfb_ext, wb, c->stream); break;
        case 5: r = run_traces_vjp<5>(c, wfb, wfb_ext, wb, c->stream); break;
        case 6: r = run_traces_vjp<6>(c, wfb, wfb_ext, wb, c->stream); break;
    }
    return acheck(c, r, "traces_vjp");
}

kbl_status kbl_rhs_vjp(kbl_ctx* c, const double* w, const double* wf, const double* Rb, double* wb, double* wfb,
                       double* wfb_ext)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (c->phys.flux != 0) return afail(c, KBL_EINVAL, "the residual adjoint covers the Rusanov flux");
    if (c->E > 0 && (!w || !wf || !Rb || !wb || !wfb || !wfb_ext)) return afail(c, KBL_EINVAL, "null array");
    int r = -1;
    switch (c->ops.n) {
        case 2: r = run_rhs_vjp<2>(c, w, wf, Rb, wb, wfb, wfb_ext, c->stream); break;
        case 3: r = run_rhs_vjp<3>(c, w, wf, Rb, wb, wfb, wfb_ext, c->stream); break;
        case 4: r = run_rhs_vjp<4>(c, w, wf, Rb, wb, wfb, wfb_ext, c->stream); break;
        case 5: r = run_rhs_vjp<5>(c, w, wf, Rb, wb, wfb, wfb_ext, c->stream); break;
        case 6: r = run_rhs_vjp<6>(c, w, wf, Rb, wb, wfb, wfb_ext, c->stream); break;
    }
    return acheck(c, r, "rhs_vjp");
}

kbl_status kbl_bounds_vjp(kbl_ctx* c, const double* w, const double* wf, const double* bnd, const double* bndb,
                          double* wb, double* wfb, double* wfb_ext)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (!adj_grid_ok(c)) return afail(c, KBL_EINVAL, "the bounds adjoint covers the trapezoidal rule on 8, 16, 32 or 64 nodes per axis");
    if (c->E > 0 && (!w || !wf || !bnd || !bndb || !wb || !wfb || !wfb_ext))
        return afail(c, KBL_EINVAL, "null array");
    int r = -1;
    switch (c->ops.n) {
        case 2: r = run_bounds_vjp<2>(c, w, wf, bnd, bndb, wb, wfb, wfb_ext, c->stream); break;
        case 3: r = run_bounds_vjp<3>(c, w, wf, bnd, bndb, wb, wfb, wfb_ext, c->stream); break;
        case 4: r = run_bounds_vjp<4>(c, w, wf, bnd, bndb, wb, wfb, wfb_ext, c->stream); break;
        case 5: r = run_bounds_vjp<5>(c, w, wf, bnd, bndb, wb, wfb, wfb_ext, c->stream); break;
        case 6: r = run_bounds_vjp<6>(c, w, wf, bnd, bndb, wb, wfb, wfb_ext, c->stream); break;
    }
    return acheck(c, r, "bounds_vjp");
}

kbl_status kbl_stage_vjp(kbl_ctx* c, int s, double dt, const double* wn, const double* ws, const double* R,
                         const double* bnd, const double* ob, int accumulate_wn, double* wnb, double* wsb,
                         double* Rb, double* bndb)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (s < 0 || s > 2) return afail(c, KBL_EINVAL, "stage must be 0, 1 or 2");
    if (c->E > 0 && (!wn || !ws || !R || !bnd || !ob || !wnb || !wsb || !Rb || !bndb))
        return afail(c, KBL_EINVAL, "null array");
    int r = -1;
    switch (c->ops.n) {
        case 2: r = run_stage_vjp<2>(c, s, dt, wn, ws, R, bnd, ob, accumulate_wn, wnb, wsb, Rb, bndb, c->stream); break;
        case 3: r = run_stage_vjp<3>(c, s, dt, wn, ws, R, bnd, ob, accumulate_wn, wnb, wsb, Rb, bndb, c->stream); break;
        case 4: r = run_stage_vjp<4>(c, s, dt, wn, ws, R, bnd, ob, accumulate_wn, wnb, wsb, Rb, bndb, c->stream); break;
        case 5: r = run_stage_vjp<5>(c, s, dt, wn, ws, R, bnd, ob, accumulate_wn, wnb, wsb, Rb, bndb, c->stream); break;
        case 6: r = run_stage_vjp<6>(c, s, dt, wn, ws, R, bnd, ob, accumulate_wn, wnb, wsb, Rb, bndb, c->stream); break;
    }
    return acheck(c, r, "stage_vjp");
}

kbl_status kbl_entropy(kbl_ctx* c, const double* w, double* J_dev)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (!J_dev || (c->E > 0 && !w)) return afail(c, KBL_EINVAL, "null array");
    const size_t nb = ((size_t)c->E * c->ns + NT_ENT - 1) / NT_ENT;
    if (c->ent_cap < nb + 1) {
        cudaStreamSynchronize(c->stream);
        if (c->d_ent) cudaFree(c->d_ent);
        c->d_ent = nullptr;
        c->ent_cap = 0;
        if (cudaMalloc((void**)&c->d_ent, (nb + 1) * sizeof(double)) != cudaSuccess)
            return afail(c, KBL_ENOMEM, "entropy scratch");
        c->ent_cap = nb + 1;
    }
    int r = -1;
    switch (c->ops.n) {
        case 2: r = run_entropy<2>(c, w, c->d_ent, J_dev, c->stream); break;
        case 3: r = run_entropy<3>(c, w, c->d_ent, J_dev, c->stream); break;
        case 4: r = run_entropy<4>(c, w, c->d_ent, J_dev, c->stream); break;
        case 5: r = run_entropy<5>(c, w, c->d_ent, J_dev, c->stream); break;
        case 6: r = run_entropy<6>(c, w, c->d_ent, J_dev, c->stream); break;
    }
    return acheck(c, r, "entropy");
}

kbl_status kbl_entropy_vjp(kbl_ctx* c, const double* w, double Jb, double* wb)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (c->E > 0 && (!w || !wb)) return afail(c, KBL_EINVAL, "null array");
    int r = -1;
    switch (c->ops.n) {
        case 2: r = run_entropy_vjp<2>(c, w, Jb, wb, c->stream); break;
        case 3: r = run_entropy_vjp<3>(c, w, Jb, wb, c->stream); break;
        case 4: r = run_entropy_vjp<4>(c, w, Jb, wb, c->stream); break;
        case 5: r = run_entropy_vjp<5>(c, w, Jb, wb, c->stream); break;
        case 6: r = run_entropy_vjp<6>(c, w, Jb, wb, c->stream); break;
    }
    return acheck(c, r, "entropy_vjp");
}

kbl_status kbl_step_fixed(kbl_ctx* c, double* w, double dt)
{
    return kbl_forward_segment(c, w, &dt, 1, nullptr);
}

kbl_status kbl_forward_segment(kbl_ctx* c, double* w, const double* dts, int n, double* bnd_out)
{
    if (!c || !c->mesh_ready) return afail(c, KBL_ESTATE, "no mesh");
    if (n < 0 || (n > 0 && !dts) || (c->E > 0 && !w)) return afail(c, KBL_EINVAL, "bad argument");
    for (int k = 0; k < n; k++)
        if (!(dts[k] >= 0.0)) return afail(c, KBL_EINVAL, "negative or NaN dt");
    if (c->E == 0 || n == 0) return KBL_OK;
    const size_t B = (size_t)2 * c->nv * c->E;
    int launches = 0;
    for (int k = 0; k < n; k++) {
        k_set_scalar<<<1, 1, 0, c->stream>>>(c->d_scal, dts[k]);
        const int r = issue_fixed(c, w, c->d_scal, bnd_out ? bnd_out + (size_t)k * 3 * B : nullptr, c->stream);
        if (r < 0) return afail(c, KBL_EINVAL, "order/dimension not compiled in");
        launches += r + 1;
    }
    return acheck(c, launches, "forward_segment");
}

kbl_status kbl_adjoint_step(kbl_ctx* c, const double* w, double dt, double* wbar)
{
    return kbl_adjoint_segment(c, w, &dt, 1, nullptr, wbar);
}

kbl_status kbl_adjoint_segment(kbl_ctx* c, const double* w0, const double* dts, int n, const double* bnd_in,
                               double* wbar)
{
    if (!adj_ok(c)) return afail(c, KBL_ESTATE, "no 2D mesh");
    if (!adj_grid_ok(c)) return afail(c, KBL_EINVAL, "the bounds adjoint covers the trapezoidal rule on 8, 16, 32 or 64 nodes per axis");
    if (c->cfg.precision != KBL_FP64) return afail(c, KBL_EINVAL, "the adjoint runs in FP64");
    if (c->phys.flux != 0) return afail(c, KBL_EINVAL, "the residual adjoint covers the Rusanov flux");
    if (n < 0 || (n > 0 && !dts) || (c->E > 0 && (!w0 || !wbar))) return afail(c, KBL_EINVAL, "bad argument");
    for (int k = 0; k < n; k++)
        if (!(dts[k] >= 0.0)) return afail(c, KBL_EINVAL, "negative or NaN dt");
    if (c->E == 0 || n == 0) return KBL_OK;
    kbl_status st = adj_reserve(c, n);
    if (st != KBL_OK) return st;
    const int r = issue_segment(c, w0, dts, n, bnd_in, wbar, c->stream);
    if (r < 0) return afail(c, KBL_EINVAL, "order / velocity grid not compiled in");
    return acheck(c, r, "adjoint_segment");
}

}  // extern "C"
