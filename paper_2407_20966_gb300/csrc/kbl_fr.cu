// kbl_fr.cu -- flux-reconstruction kernels: face traces, stencil gather, the FR
// residual with Rusanov interface fluxes, and the device-side time step.
//
// Scheme (Sec. 2.3 and Sec. 5 of the paper): Gauss-Legendre solution and flux
// points on axis-aligned lines/quads, Huynh's FR with the g_DG correction
// (which recovers nodal DG), Rusanov common fluxes (assumption (iv), Sec. 4).
#include <cfloat>

#include "kbl_fr_body.cuh"

namespace {

// ---------------------------------------------------------------------------
// traces: wf[v][e][fp] = sum_i l_i(+-1) w[v][e][line(fp, i)]
// One thread per (element, face point); the interpolation weights are uniform
// across the warp, so they are read from the parameter block.  T is the
// arithmetic type (double for the FP64 path, float for the FP32-mixed path);
// storage is FP64 in both.
// ---------------------------------------------------------------------------
template <int DIM, int N, typename T>
__global__ void __launch_bounds__(256) k_traces(const double* __restrict__ w, double* __restrict__ wf,
                                                int E, FrOps ops)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    kbl_grid_dep_sync();
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
        T s = T(0);
#pragma unroll
        for (int i = 0; i < N; i++) {
            const T l = (T)(plus ? ops.lp[i] : ops.lm[i]);
            const int nd = along_x ? k * N + i : i * N + k;
            s += l * (T)we[(DIM == 1) ? i : nd];
        }
        wf[((size_t)v * E + e) * NFP + fp] = (double)s;
    }
}

template <int DIM, int N>
int run_traces(const kbl_ctx* c, const double* w, double* wf, cudaStream_t s)
{
    const size_t total = (size_t)c->E * kbl_nfp<DIM>(N);
    if (total == 0) return 0;
    const int bs = 256;
    const unsigned grid = (unsigned)((total + bs - 1) / bs);
    // FP64 in both precision modes: converting each input to FP32 costs an FP64-pipe slot
    // on GB300, as much as the FP64 multiply-add it would replace.
    kbl_launch(k_traces<DIM, N, double>, grid, bs, 0, s, c->pdl, w, wf, c->E, c->ops);
    return 1;
}

// ---------------------------------------------------------------------------
// gather: S[e - e0][r][v] for the stencil rows of kbl.h (plain copies)
// ---------------------------------------------------------------------------
template <int DIM, int N, bool WIDE = false>
__global__ void k_gather(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m,
                         int e0, int n, double* __restrict__ S)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NST = WIDE ? 3 * NS : NS + 2 * NFP;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * NST * NV) return;
    const int v = (int)(t % NV);
    const int r = (int)((t / NV) % NST);
    const int e = e0 + (int)(t / ((size_t)NV * NST));
    double val;
    if (WIDE) val = kbl_wide1d<N>(w, m, e, r, v);
    else if (r < NS) val = w[((size_t)v * m.E + e) * NS + r];
    else if (r < NS + NFP) val = wf[((size_t)v * m.E + e) * NFP + (r - NS)];
    else val = kbl_exterior<DIM, N>(wf, m, e, r - NS - NFP, v);
    S[t] = val;
}

template <int DIM, int N>
int run_gather(const kbl_ctx* c, const double* w, const double* wf, int e0, int n, double* S,
               cudaStream_t s)
{
    const bool wide = DIM == 1 && c->cfg.stencil == 1;
    const int NST = wide ? 3 * kbl_ns<DIM>(N) : kbl_ns<DIM>(N) + 2 * kbl_nfp<DIM>(N);
    const size_t total = (size_t)n * NST * (DIM + 2);
    if (total == 0) return 0;
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (wide) k_gather<DIM, N, true><<<grid, 256, 0, s>>>(w, wf, mesh_of(c), e0, n, S);
    else k_gather<DIM, N, false><<<grid, 256, 0, s>>>(w, wf, mesh_of(c), e0, n, S);
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
    static constexpr int NS = kbl_ns<DIM>(N);
    static constexpr int EPB = (DIM == 1) ? 32 : 8;
    static constexpr int NT = EPB * NS;
};

#ifdef KBL_RHS_MINB
#define KBL_RHS_BOUNDS(...) __launch_bounds__(__VA_ARGS__, KBL_RHS_MINB)
#else
#define KBL_RHS_BOUNDS(...) __launch_bounds__(__VA_ARGS__)
#endif
template <int DIM, int N, typename T>
__global__ void KBL_RHS_BOUNDS(RhsShape<DIM, N>::NT)
k_rhs(const double* __restrict__ w, const double* __restrict__ wf, MeshDev m, FrOps ops,
      double gamma_d, double* __restrict__ R, int flux)
{
    using SH = RhsShape<DIM, N>;
    kbl_grid_dep_sync();
    __shared__ kbl_dev::RhsSmem<DIM, N, T, SH::EPB> sm;
    kbl_dev::rhs_block<DIM, N, T, SH::EPB>(sm, SH::NT, w, wf, m, ops, gamma_d, R, blockIdx.x * SH::EPB, SH::EPB,
                                            flux);
}

template <int DIM, int N>
int run_rhs(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s)
{
    using SH = RhsShape<DIM, N>;
    if (c->E == 0) return 0;
    const unsigned grid = (unsigned)((c->E + SH::EPB - 1) / SH::EPB);
    if (c->cfg.precision == KBL_FP32_MIXED)
        kbl_launch(k_rhs<DIM, N, float>, grid, SH::NT, 0, s, c->pdl, w, wf, mesh_of(c), c->ops, c->phys.gamma, R,
                   c->phys.flux);
    else
        kbl_launch(k_rhs<DIM, N, double>, grid, SH::NT, 0, s, c->pdl, w, wf, mesh_of(c), c->ops, c->phys.gamma, R,
                   c->phys.flux);
    return 1;
}

// ---------------------------------------------------------------------------
// Time step: dtbits <- min over points and axes of cfl * h / (|U| + c), as the
// bit pattern of a positive double (integer order = value order), then the
// finalize kernel clips to the end time.
// ---------------------------------------------------------------------------
template <int DIM, int N, typename T>
__global__ void __launch_bounds__(256) k_dt(const double* __restrict__ w, MeshDev m, double gamma_d,
                                            double cfl, unsigned long long* dtbits)
{
    constexpr int NS = kbl_ns<DIM>(N), NV = DIM + 2;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double best = DBL_MAX;
    if (t < (size_t)m.E * NS) {
        const int e = (int)(t / NS), nd = (int)(t % NS);
        const T gamma = (T)gamma_d;
        T q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) q[v] = kbl_dev::from_f64<T>(w[((size_t)v * m.E + e) * NS + nd]);
        const T P = kbl_pressure<DIM, T>(q, gamma - T(1));
        const T a = sqrt(gamma * P / q[0]);
        T b = (T)DBL_MAX;
        if (sizeof(T) == sizeof(float)) b = (T)FLT_MAX;
#pragma unroll
        for (int k = 0; k < DIM; k++) {
            const T cand = (T)cfl * (kbl_dev::from_f64<T>(m.h[e * DIM + k]) / (fabs(q[1 + k] / q[0]) + a));
            b = fmin(b, cand);
        }
        best = kbl_dev::to_f64<T>(b);
    }
    unsigned long long bits = __double_as_longlong(best);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = ob < bits ? ob : bits;
    }
    // one atomic per block: thousands of warps on one address would serialise in L2
    __shared__ unsigned long long swarp[8];
    if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) bits = swarp[k] < bits ? swarp[k] : bits;
        atomicMin(dtbits, bits);
    }
}

__global__ void k_dt_finalize(unsigned long long* dtbits, const double* scal, double* dt_out,
                              int clip)
{
    // scal: [0] dt, [1] t, [2] t_end.  With clip the step stops at t_end.  The reduction word is
    // left at its start value, which the fused traces + time step kernel of kbl_step relies on.
    double dt = __longlong_as_double((long long)*dtbits);
    *dtbits = 0x7f7f7f7f7f7f7f7full;
    if (!(dt > 0.0) || !(dt < DBL_MAX)) dt = 0.0;
    if (clip) dt = fmin(dt, scal[2] - scal[1]);
    *dt_out = dt;
}

__global__ void k_time_advance(double* scal) { scal[1] += scal[0]; }

// ---------------------------------------------------------------------------
// The first work of a step in one pass over w: the face traces (as k_traces, FP64) and the time
// step (as k_dt with its arithmetic type T), whose block minima meet in dtbits; the last block to
// finish (a counter of finished blocks) decodes the step, clips it to the end time and resets the
// reduction word and the counter for the next step, so that neither a memset nor a finalizing
// kernel is needed.  TRACES = false: the time step alone (one thread per solution point), for
// a step graph that runs it on a branch beside k_traces: only the stage kernels read it.
// ---------------------------------------------------------------------------
template <int DIM, int N, typename T, bool TRACES = true>
__global__ void __launch_bounds__(256) k_traces_dt(const double* __restrict__ w, double* __restrict__ wf, MeshDev m,
                                                   FrOps ops, double gamma_d, double cfl,
                                                   unsigned long long* dtbits, unsigned* blocks_done, double* scal)
{
    constexpr int NS = kbl_ns<DIM>(N), NFP = kbl_nfp<DIM>(N), NV = DIM + 2;
    constexpr int NK = (TRACES && NFP > NS) ? NFP : NS;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = t < (size_t)m.E * NK;
    const int e = in ? (int)(t / NK) : 0, k = (int)(t % NK);
    if (TRACES && in && k < NFP) {   // traces: the operations and order of k_traces
        const int fp = k;
        const int f = (DIM == 1) ? fp : fp / N;
        const int kk = (DIM == 1) ? 0 : fp % N;
        const bool plus = f & 1;
        const bool along_x = (DIM == 1) || f < 2;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double* we = w + ((size_t)v * m.E + e) * NS;
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) {
                const double l = plus ? ops.lp[i] : ops.lm[i];
                const int nd = along_x ? kk * N + i : i * N + kk;
                s += l * we[(DIM == 1) ? i : nd];
            }
            wf[((size_t)v * m.E + e) * NFP + fp] = s;
        }
    }
    double best = DBL_MAX;
    if (in && k < NS) {    // time step: the operations of k_dt
        const int nd = k;
        const T gamma = (T)gamma_d;
        T q[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) q[v] = kbl_dev::from_f64<T>(w[((size_t)v * m.E + e) * NS + nd]);
        const T P = kbl_pressure<DIM, T>(q, gamma - T(1));
        const T a = sqrt(gamma * P / q[0]);
        T b = (T)DBL_MAX;
        if (sizeof(T) == sizeof(float)) b = (T)FLT_MAX;
#pragma unroll
        for (int kd = 0; kd < DIM; kd++) {
            const T cand = (T)cfl * (kbl_dev::from_f64<T>(m.h[e * DIM + kd]) / (fabs(q[1 + kd] / q[0]) + a));
            b = fmin(b, cand);
        }
        best = kbl_dev::to_f64<T>(b);
    }
    unsigned long long bits = __double_as_longlong(best);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = ob < bits ? ob : bits;
    }
    __shared__ unsigned long long swarp[8];
    __shared__ int s_last;
    if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) bits = swarp[q] < bits ? swarp[q] : bits;
        atomicMin(dtbits, bits);
        __threadfence();
        s_last = atomicAdd(blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long fb = atomicAdd(dtbits, 0ull);
        double dt = __longlong_as_double((long long)fb);
        if (!(dt > 0.0) || !(dt < DBL_MAX)) dt = 0.0;
        scal[0] = fmin(dt, scal[2] - scal[1]);   // clipped to the end time
        *dtbits = 0x7f7f7f7f7f7f7f7full;         // the value the reduction starts from
        *blocks_done = 0u;
    }
}

template <int DIM, int N>
int run_dt(const kbl_ctx* c, const double* w, double cfl, double* dt_out, int clip, cudaStream_t s)
{
    cudaMemsetAsync(c->d_dtbits, 0x7f, sizeof(unsigned long long), s);
    int n = 0;
    const size_t total = (size_t)c->E * kbl_ns<DIM>(N);
    if (total > 0) {
        const unsigned grid = (unsigned)((total + 255) / 256);
        if (c->cfg.precision == KBL_FP32_MIXED)
            k_dt<DIM, N, float><<<grid, 256, 0, s>>>(w, mesh_of(c), c->phys.gamma, cfl, c->d_dtbits);
        else
            k_dt<DIM, N, double><<<grid, 256, 0, s>>>(w, mesh_of(c), c->phys.gamma, cfl, c->d_dtbits);
        n++;
    }
    k_dt_finalize<<<1, 1, 0, s>>>(c->d_dtbits, c->d_scal, dt_out, clip);
    return n + 1;
}

template <int DIM, int N>
int run_traces_dt(const kbl_ctx* c, const double* w, double* wf, double cfl, cudaStream_t s)
{
    constexpr int NK = kbl_ns<DIM>(N) > kbl_nfp<DIM>(N) ? kbl_ns<DIM>(N) : kbl_nfp<DIM>(N);
    const size_t total = (size_t)c->E * NK;
    if (total == 0) return 0;
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (c->cfg.precision == KBL_FP32_MIXED)
        k_traces_dt<DIM, N, float><<<grid, 256, 0, s>>>(w, wf, mesh_of(c), c->ops, c->phys.gamma, cfl, c->d_dtbits,
                                                        c->d_blocks_done, c->d_scal);
    else
        k_traces_dt<DIM, N, double><<<grid, 256, 0, s>>>(w, wf, mesh_of(c), c->ops, c->phys.gamma, cfl, c->d_dtbits,
                                                         c->d_blocks_done, c->d_scal);
    return 1;
}

// The time step of k_traces_dt alone: the same per-node arithmetic and the same exact minimum,
// so the same dt bit for bit.
template <int DIM, int N>
int run_dt_step(const kbl_ctx* c, const double* w, double cfl, cudaStream_t s)
{
    const size_t total = (size_t)c->E * kbl_ns<DIM>(N);
    if (total == 0) return 0;
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (c->cfg.precision == KBL_FP32_MIXED)
        k_traces_dt<DIM, N, float, false><<<grid, 256, 0, s>>>(w, nullptr, mesh_of(c), c->ops, c->phys.gamma, cfl,
                                                               c->d_dtbits, c->d_blocks_done, c->d_scal);
    else
        k_traces_dt<DIM, N, double, false><<<grid, 256, 0, s>>>(w, nullptr, mesh_of(c), c->ops, c->phys.gamma, cfl,
                                                                c->d_dtbits, c->d_blocks_done, c->d_scal);
    return 1;
}

}  // namespace

int launch_traces_dt(const kbl_ctx* c, const double* w, double* wf, double cfl, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_traces_dt, c, w, wf, cfl, s);
}

int launch_dt_step(const kbl_ctx* c, const double* w, double cfl, cudaStream_t s)
{
    KBL_DISPATCH(c->cfg.dim, c->cfg.p + 1, run_dt_step, c, w, cfl, s);
}

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
    const int r = launch_rhs_tc(c, w, wf, R, s);
    if (r >= 0) return r;
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
