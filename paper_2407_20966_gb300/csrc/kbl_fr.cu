// kbl_fr.cu -- flux-reconstruction kernels: face traces, stencil gather, the FR
// residual with Rusanov interface fluxes, and the device-side time step.
//
// Scheme (Sec. 2.3 and Sec. 5 of the paper): Gauss-Legendre solution and flux
// points on axis-aligned lines/quads, Huynh's FR with the g_DG correction
// (which recovers nodal DG), Rusanov common fluxes (assumption (iv), Sec. 4).
#include <cfloat>

#include "kbl_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// traces: wf[v][e][fp] = sum_i l_i(+-1) w[v][e][line(fp, i)]
// One thread per (element, face point); the interpolation weights are uniform
// across the warp, so they are read from the parameter block.
// ---------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_traces(const double* __restrict__ w, double* __restrict__ wf,
                                                int E, FrOps ops)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)E * NFP) return;
    const int e = (int)(t / NFP), fp = (int)(t % NFP);
    const int f = (DIM == 1) ? fp : fp / N;
    const int k = (DIM == 1) ? 0 : fp % N;
    const bool plus = f & 1;
    const bool along_x = (DIM == 1) || f < 2;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const double* we = w + ((size_t)v * E + e) * NS;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; i++) {
            const double l = plus ? ops.lp[i] : ops.lm[i];
            const int nd = along_x ? k * N + i : i * N + k;
            s += l * we[(DIM == 1) ? i : nd];
        }
        wf[((size_t)v * E + e) * NFP + fp] = s;
    }
}

template <int DIM, int N>
int run_traces(const kbl_ctx* c, const double* w, double* wf, cudaStream_t s)
{
    const size_t total = (size_t)c->E * kbl_nfp<DIM>(N);
    if (total == 0) return 0;
    const int bs = 256;
    k_traces<DIM, N><<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(w, wf, c->E, c->ops);
    return 1;
}

// ---------------------------------------------------------------------------
// gather: S[e - e0][r][v] for the stencil rows of kbl.h (plain copies)
// ---------------------------------------------------------------------------
template <int DIM, int N>
__global__ void k_gather(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m,
                         int e0, int n, double* __restrict__ S)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NST = NS + 2 * NFP;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * NST * NV) return;
    const int v = (int)(t % NV);
    const int r = (int)((t / NV) % NST);
    const int e = e0 + (int)(t / ((size_t)NV * NST));
    double val;
    if (r < NS) val = w[((size_t)v * m.E + e) * NS + r];
    else if (r < NS + NFP) val = wf[((size_t)v * m.E + e) * NFP + (r - NS)];
    else val = kbl_exterior<DIM, N>(wf, m, e, r - NS - NFP, v);
    S[t] = val;
}

template <int DIM, int N>
int run_gather(const kbl_ctx* c, const double* w, const double* wf, int e0, int n, double* S,
               cudaStream_t s)
{
    constexpr int NST = kbl_ns<DIM>(N) + 2 * kbl_nfp<DIM>(N);
    const size_t total = (size_t)n * NST * (DIM + 2);
    if (total == 0) return 0;
    k_gather<DIM, N><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(w, wf, mesh_of(c), e0, n, S);
    return 1;
}

// ---------------------------------------------------------------------------
// FR residual.  A block holds EPB elements, one thread per solution point.
//   1. states and physical fluxes at the solution points -> shared memory
//   2. per face point: Rusanov flux of (interior trace, exterior value) minus
//      the interpolated discontinuous flux -> jump J
//   3. per solution point and axis: D F + g_L' J_minus + g_R' J_plus,
//      R = -sum_axes (2 / h_axis) dF/dxi
// ---------------------------------------------------------------------------
template <int DIM, int N>
struct RhsShape {
    static constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    static constexpr int EPB = (DIM == 1) ? 32 : 8;
    static constexpr int NT = EPB * NS;
};

template <int DIM, int N>
__global__ void __launch_bounds__(RhsShape<DIM, N>::NT)
k_rhs(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, FrOps ops,
      double gamma, double* __restrict__ R)
{
    using SH = RhsShape<DIM, N>;
    constexpr int NS = SH::NS, NFP = SH::NFP, NV = SH::NV, EPB = SH::EPB, NT = SH::NT;
    constexpr int NFPF = (DIM == 1) ? 1 : N;
    __shared__ double sF[EPB][DIM][NV][NS];
    __shared__ double sJ[EPB][NFP][NV];
    __shared__ double sD[N][N], sgl[N], sgr[N], slm[N], slp[N];

    const int tid = threadIdx.x;
    for (int i = tid; i < N * N; i += NT) sD[i / N][i % N] = ops.D[i / N][i % N];
    if (tid < N) {
        sgl[tid] = ops.gl[tid];
        sgr[tid] = ops.gr[tid];
        slm[tid] = ops.lm[tid];
        slp[tid] = ops.lp[tid];
    }
    const int el = tid / NS, nd = tid % NS;
    const int e = blockIdx.x * EPB + el;
    const double gm1 = gamma - 1.0;
    if (e < m.E) {
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) q[v] = w[((size_t)v * m.E + e) * NS + nd];
#pragma unroll
        for (int dir = 0; dir < DIM; dir++) {
            double F[NV];
            kbl_flux<DIM>(q, dir, gm1, F);
#pragma unroll
            for (int v = 0; v < NV; v++) sF[el][dir][v][nd] = F[v];
        }
    }
    __syncthreads();
    for (int t = tid; t < EPB * NFP; t += NT) {
        const int ell = t / NFP, fp = t % NFP;
        const int ee = blockIdx.x * EPB + ell;
        if (ee >= m.E) continue;
        const int f = fp / NFPF, k = fp % NFPF, dir = f >> 1, side = f & 1;
        double qi[NV], qe[NV], Fc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            qi[v] = wf[((size_t)v * m.E + ee) * NFP + fp];
            qe[v] = kbl_exterior<DIM, N>(wf, m, ee, fp, v);
        }
        if (side == 0) kbl_rusanov<DIM>(qe, qi, dir, gamma, Fc);
        else kbl_rusanov<DIM>(qi, qe, dir, gamma, Fc);
        const double* l = side ? slp : slm;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double FD = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int node = (DIM == 1) ? i : (dir == 0 ? k * N + i : i * N + k);
                FD += l[i] * sF[ell][dir][v][node];
            }
            sJ[ell][fp][v] = Fc[v] - FD;
        }
    }
    __syncthreads();
    if (e >= m.E) return;
    const int i = (DIM == 1) ? nd : nd % N;
    const int j = (DIM == 1) ? 0 : nd / N;
    const double sx = 2.0 / m.h[e * DIM + 0];
    const double sy = (DIM == 2) ? 2.0 / m.h[e * DIM + 1] : 0.0;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        double dx = 0.0;
#pragma unroll
        for (int mm = 0; mm < N; mm++) dx += sD[i][mm] * sF[el][0][v][(DIM == 1) ? mm : j * N + mm];
        dx += sgl[i] * sJ[el][0 * NFPF + j][v] + sgr[i] * sJ[el][1 * NFPF + j][v];
        double r = -sx * dx;
        if (DIM == 2) {
            double dy = 0.0;
#pragma unroll
            for (int mm = 0; mm < N; mm++) dy += sD[j][mm] * sF[el][DIM - 1][v][mm * N + i];
            dy += sgl[j] * sJ[el][2 * NFPF + i][v] + sgr[j] * sJ[el][3 * NFPF + i][v];
            r -= sy * dy;
        }
        R[((size_t)v * m.E + e) * NS + nd] = r;
    }
}

template <int DIM, int N>
int run_rhs(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s)
{
    using SH = RhsShape<DIM, N>;
    if (c->E == 0) return 0;
    const unsigned grid = (unsigned)((c->E + SH::EPB - 1) / SH::EPB);
    k_rhs<DIM, N><<<grid, SH::NT, 0, s>>>(w, wf, mesh_of(c), c->ops, c->phys.gamma, R);
    return 1;
}

// ---------------------------------------------------------------------------
// Time step: dtbits <- min over points and axes of cfl * h / (|U| + c), as the
// bit pattern of a positive double (integer order = value order), then the
// finalize kernel clips to the end time.
// ---------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_dt(const double* __restrict__ w, MeshDev m, double gamma,
                                            double cfl, unsigned long long* dtbits)
{
    constexpr int NS = kbl_ns<DIM>(N), NV = DIM + 2;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double best = DBL_MAX;
    if (t < (size_t)m.E * NS) {
        const int e = (int)(t / NS), nd = (int)(t % NS);
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) q[v] = w[((size_t)v * m.E + e) * NS + nd];
        const double P = kbl_pressure<DIM>(q, gamma - 1.0);
        const double a = sqrt(gamma * P / q[0]);
#pragma unroll
        for (int k = 0; k < DIM; k++) {
            const double cand = cfl * (m.h[e * DIM + k] / (fabs(q[1 + k] / q[0]) + a));
            best = fmin(best, cand);
        }
    }
    unsigned long long b = __double_as_longlong(best);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
        b = ob < b ? ob : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(dtbits, b);
}

__global__ void k_dt_finalize(const unsigned long long* dtbits, const double* scal, double* dt_out,
                              int clip)
{
    // scal: [0] dt, [1] t, [2] t_end.  With clip the step stops at t_end.
    double dt = __longlong_as_double((long long)*dtbits);
    if (!(dt > 0.0) || !(dt < DBL_MAX)) dt = 0.0;
    if (clip) dt = fmin(dt, scal[2] - scal[1]);
    *dt_out = dt;
}

__global__ void k_time_advance(double* scal) { scal[1] += scal[0]; }

template <int DIM, int N>
int run_dt(const kbl_ctx* c, const double* w, double cfl, double* dt_out, int clip, cudaStream_t s)
{
    cudaMemsetAsync(c->d_dtbits, 0x7f, sizeof(unsigned long long), s);
    int n = 0;
    const size_t total = (size_t)c->E * kbl_ns<DIM>(N);
    if (total > 0) {
        k_dt<DIM, N><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(w, mesh_of(c), c->phys.gamma, cfl,
                                                                    c->d_dtbits);
        n++;
    }
    k_dt_finalize<<<1, 1, 0, s>>>(c->d_dtbits, c->d_scal, dt_out, clip);
    return n + 1;
}

}  // namespace

MeshDev mesh_of(const kbl_ctx* c)
{
    MeshDev m;
    m.E = c->E;
    m.nbr = c->d_nbr;
    m.h = c->d_h;
    m.bc = c->d_bc;
    m.n_bc = c->n_bc;
    return m;
}

int launch_traces(const kbl_ctx* c, const double* w, double* wf, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_traces, c, w, wf, s);
}

int launch_gather(const kbl_ctx* c, const double* w, const double* wf, int e0, int n, double* S,
                  cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_gather, c, w, wf, e0, n, S, s);
}

int launch_rhs(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_rhs, c, w, wf, R, s);
}

int launch_dt(const kbl_ctx* c, const double* w, double cfl, double* dt_out, int clip, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_dt, c, w, cfl, dt_out, clip, s);
}

int launch_time_advance(const kbl_ctx* c, cudaStream_t s)
{
    k_time_advance<<<1, 1, 0, s>>>(c->d_scal);
    return 1;
}
