// kbl_internal.cuh -- shared declarations of the libkbl CUDA sources.
//
// Layout and indexing conventions are those of include/kbl.h.  Everything here
// is internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "kbl.h"

#define KBL_PMAX 5
#define KBL_NMAX (KBL_PMAX + 1)

// Reference-element FR operators of one order, passed to kernels by value.
struct FrOps {
    int n;                                  // p + 1
    double x[KBL_NMAX], wq[KBL_NMAX];       // Gauss-Legendre nodes, weights
    double lm[KBL_NMAX], lp[KBL_NMAX];      // l_i(-1), l_i(+1)
    double D[KBL_NMAX][KBL_NMAX];           // D[i][m] = l_m'(x_i)
    double gl[KBL_NMAX], gr[KBL_NMAX];      // g_L'(x_i), g_R'(x_i)
    // limiter constants, computed on the host once per order: the 2D mean weights
    // wq[n % N] wq[n / N], 1 / sum of the weights in 1D and 2D, and Lambda = max over the two
    // ends of sum_i |l_i(+-1)| (a face value lies within Lambda max_i |w_i - mean| of the mean)
    double wm2[KBL_NMAX * KBL_NMAX];
    double winv1, winv2, lam;
    // FP32 copies (rounded on the host) of the residual's operators, for the FP32 arithmetic
    float Df[KBL_NMAX][KBL_NMAX], glf[KBL_NMAX], grf[KBL_NMAX], lmf[KBL_NMAX], lpf[KBL_NMAX];
    // for the FP32 screen of the limiter: the mean weights and 1 / their sum rounded to
    // nearest, and Lambda rounded up
    float wm2f[KBL_NMAX * KBL_NMAX], wqf[KBL_NMAX], winv1f, winv2f, lamf;
};

// FP32 value nearest x, moved one step up (down) when it lies below (above) x: a float
// bound of a double, for the conservative FP32 screens.
inline float kbl_f32_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}
inline float kbl_f32_down(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}

// Physical and method constants, passed by value.
struct Phys {
    double gamma, k, r_fac, eps, rho_floor, p_floor;
    int eps_rule;
    int nu[2];
    int uncoupled;
    int flux;   // 0 Rusanov, 1 HLLC, 2 HLL
    // velocity quadrature: per-node weights in units of the grid spacing (nu[0] values,
    // the same rule on every axis; qwf its FP32 copy), or nullptr for the trapezoidal rule
    const double* qw;
    const float* qwf;
    // derived on the host (kbl_phys_derive), so that FP32 kernels spend no FP64 division or
    // conversion on them: gamma - 1, k, delta / 2 = 1/(gamma - 1) - d/2 for d = 2, 1 -+ r
    float gm1f, kf, half_delta2f;
    double rel_lo, rel_hi;
    float rel_lof, rel_hif;   // FP32 copies of 1 -+ r
    // float bounds for the limiter's FP32 screen: eps and p_floor rounded up, gamma - 1 down
    float epsf_up, pfloorf_up, gm1f_down;
};

inline void kbl_phys_derive(Phys& p)
{
    p.gm1f = (float)(p.gamma - 1.0);
    p.kf = (float)p.k;
    p.half_delta2f = 0.5f * (float)(2.0 / (p.gamma - 1.0) - 2.0);
    p.epsf_up = kbl_f32_up(p.eps);
    p.pfloorf_up = kbl_f32_up(p.p_floor);
    p.gm1f_down = kbl_f32_down(p.gamma - 1.0);
    p.rel_lo = 1.0 - p.r_fac;
    p.rel_hi = 1.0 + p.r_fac;
    p.rel_lof = (float)p.rel_lo;
    p.rel_hif = (float)p.rel_hi;
}

// Programmatic dependent launch inside a step graph: a kernel of the step's main chain first
// waits until the grids it depends on have completed and their writes are visible (it reads
// their outputs and overwrites buffers they read), then lets its own dependent grid be
// launched, whose blocks take SM slots as this grid's blocks retire and wait there in turn.
// Launched without the programmatic attribute, both are no-ops.
__device__ __forceinline__ void kbl_grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void kbl_grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void kbl_grid_dep_sync()
{
    kbl_grid_dep_wait();
    kbl_grid_dep_trigger();
}

// Launch `kernel` on s; with pdl, as a programmatic dependent of the work before it on s.
template <typename... KArgs, typename... Args>
cudaError_t kbl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                       Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// FP32 approximation of a double by truncating its significand, with integer operations only
// (a conversion instruction would cost an FP64-pipe slot): |result - x| <= 2^-23 |x| for
// 2^-126 <= |x| < 2^128, 0 below that range (|error| < 2^-126), infinity above it.
__device__ __forceinline__ float f32_trunc(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e32 = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e32 <= 0) return 0.0f;
    if (e32 >= 255) return __uint_as_float((hi & 0x80000000u) | 0x7f800000u);
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e32 << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// One SSP-RK3 stage in Shu-Osher form (Sec. 5) at index g: t = ws + dt R, then t (stage 0),
// 3/4 wn + 1/4 t (stage 1) or 1/3 wn + 2/3 t (stage 2).  The FMAs are written out so that every
// kernel that forms a stage (the stage kernels, with the stage known at compile time or not, and
// the adjoint's recomputation of the forward step) gets the same bits.
__device__ __forceinline__ double kbl_ssprk3(int stage, const double* wn, const double* ws, const double* R,
                                             size_t g, double dt)
{
    const double t = fma(dt, R[g], ws[g]);
    if (stage == 0) return t;
    if (stage == 1) return fma(0.75, wn[g], 0.25 * t);
    return fma(1.0 / 3.0, wn[g], (2.0 / 3.0) * t);
}

// x > 0.0 decided on the bit pattern with integer operations (true for +inf, false for
// zeros, negatives and NaN), which keeps the test off the FP64 pipe.
__device__ __forceinline__ bool kbl_positive(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000ll;
}

// Exact FP64 value of a float, with integer operations only (subnormal floats give 0).  Normal
// numbers get the exponent rebiased; infinities and NaNs the all-ones FP64 exponent with the
// 23 significand bits moved to the top of the FP64 significand, so an infinity stays one and a
// NaN stays a NaN.  A conversion instruction, even one predicated off on the finite path,
// would hold the slow FP64 pipe (measured: 4 such instructions per warp of the FP32 residual
// kept that pipe 15% busy).
__device__ __forceinline__ double f64_widen(float x)
{
    const unsigned b = __float_as_uint(x), ex = (b >> 23) & 0xffu;
    if (ex == 0u) return 0.0;
    const unsigned e64 = ex == 255u ? 0x7ffu : ex + 896u;
    const unsigned hi = (b & 0x80000000u) | (e64 << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// FP32 weight of velocity node j (see kbl_qweight), for the FP32 kernels.
__device__ __forceinline__ float kbl_qweight_f(const Phys& ph, int j, int nu)
{
    if (j >= nu) return 0.0f;
    if (ph.qwf) return ph.qwf[j];
    return (j == 0 || j == nu - 1) ? 0.5f : 1.0f;
}

// Weight, in units of the grid spacing, of velocity node j of an axis of nu nodes: the
// uploaded rule when there is one, else the trapezoidal rule of Sec. 3.7 (1/2 at both
// ends).  Nodes j >= nu pad a kernel's tile and carry no weight.
__device__ __forceinline__ double kbl_qweight(const Phys& ph, int j, int nu)
{
    if (j >= nu) return 0.0;
    if (ph.qw) return ph.qw[j];
    return (j == 0 || j == nu - 1) ? 0.5 : 1.0;
}

// One segment [jb, je) of a Maxwellian factor on an equispaced velocity axis, FP64:
//   emit(j, scale exp(-(u_j - U)^2 / (2 theta))),  u_j = lo + j h for j < nu (the nodes j >= nu
//   of a padded tile repeat the last node),
// by a product recurrence instead of one exponential per node: with d_j = u_j - U,
//   E(j + 1) = E(j) R(j),  R(j + 1) = R(j) Q,  R(j) = exp(-h (2 d_j + h) / (2 theta)),
//   Q = exp(-h^2 / theta),
// and its mirror image to the left.  It starts at the segment node nearest U, so every ratio is
// at most 1 (up to rounding): values only shrink, an underflow to 0 is harmless and nothing
// overflows.  Each step adds a few ulp; over a 16-node segment the relative error stays
// below 1e-13.  Callers that must agree bit for bit (the forward bounds and their adjoint)
// call it with the same arguments.
template <typename Emit>
__device__ __forceinline__ void kbl_gauss_segment(double scale, double U, double th, double lo, double h, int nu,
                                                  int jb, int je, Emit emit)
{
    const double i2t = 0.5 / th;
    const int jr = min(je, nu);   // real nodes of the segment: [jb, jr)
    if (jr > jb) {
        int j0 = (int)rint((U - lo) / h);
        j0 = max(jb, min(jr - 1, j0));
        const double d0 = fma((double)j0, h, lo) - U;
        const double e0 = scale * exp(-(d0 * d0) * i2t);
        const double q = exp(-2.0 * (h * h) * i2t);
        emit(j0, e0);
        double e = e0, r = exp(-h * (2.0 * d0 + h) * i2t);
        for (int j = j0 + 1; j < jr; j++) {
            e *= r;
            r *= q;
            emit(j, e);
        }
        e = e0;
        r = exp(-h * (h - 2.0 * d0) * i2t);
        for (int j = j0 - 1; j >= jb; j--) {
            e *= r;
            r *= q;
            emit(j, e);
        }
    }
    if (je > jr) {   // padding: the last real node
        const double d = fma((double)(nu - 1), h, lo) - U;
        const double ep = scale * exp(-(d * d) * i2t);
        for (int j = max(jb, jr); j < je; j++) emit(j, ep);
    }
}

// Tile size (velocity nodes per axis) of the 2D bounds kernels that holds an axis of nu nodes.
__host__ __device__ constexpr int kbl_tile_nx(int nu) { return nu <= 8 ? 8 : nu <= 16 ? 16 : nu <= 32 ? 32 : 64; }

struct MeshDev {
    int E;
    const int* nbr;     // [E][2d]
    const double* h;    // [E][d]
    const double* bc;   // [n_bc][nv]
    int n_bc;
};

#define KBL_ALPHA_BINS 10

struct DevFlags {
    int nonphysical;
    int timeout;
    unsigned long long limited;
    unsigned long long prelimit;
    unsigned long long eps_rule;                    // components where the epsilon rule of Eq. 37 fired
    unsigned long long mean_outside;                // components whose mean lies outside [lo, hi]
    unsigned long long alpha_hist[KBL_ALPHA_BINS];  // limited elements by alpha_min, bins of width 1/10
};

// Histogram bin of a limiting factor alpha in [0, 1): floor(10 alpha), at most 9.
__device__ __forceinline__ int kbl_alpha_bin(double a)
{
    const int b = (int)(a * (double)KBL_ALPHA_BINS);
    return b < 0 ? 0 : (b >= KBL_ALPHA_BINS ? KBL_ALPHA_BINS - 1 : b);
}

struct kbl_ctx {
    kbl_config cfg;
    Phys phys;
    FrOps ops;
    cudaStream_t stream = nullptr;
    int nv = 0, ns = 0, nfp = 0, nsten = 0;
    int E = 0, n_bc = 0;
    bool mesh_ready = false;
    // mesh copy
    int* d_nbr = nullptr;
    double* d_h = nullptr;
    double* d_bc = nullptr;
    // scratch
    double* d_wf = nullptr;     // [nv][E][Nfp]
    double* d_R = nullptr;      // [nv][E][Ns]
    double* d_bnd = nullptr;    // [2][nv][E]
    double* d_wa = nullptr;     // stage buffers [nv][E][Ns]
    double* d_wb = nullptr;
    double* d_whost = nullptr;  // device copy used by kbl_run_host
    double* d_whost2 = nullptr; // second device copy of kbl_run_host_ensemble (first call allocates it)
    double* d_scal = nullptr;   // [0] dt, [1] t, [2] t_end, [3] start time of kbl_run_host_ensemble
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;   // copy streams of kbl_run_host_ensemble
    cudaEvent_t ev_h2d[2] = {nullptr, nullptr}, ev_step[2] = {nullptr, nullptr}, ev_d2h[2] = {nullptr, nullptr};
    unsigned long long* d_dtbits = nullptr;
    unsigned* d_blocks_done = nullptr;   // finished-block counter of the fused traces + time step
    DevFlags* d_flags = nullptr;
    double* d_qw = nullptr;     // velocity quadrature weights (Romberg), or nullptr
    float* d_tcop = nullptr;    // split residual operator of the tensor-core residual, or nullptr
    int rhs_tc = 0;             // knob: 1 residual products on the tensor cores where covered, 0 CUDA cores
    int overlap_rhs = 1;        // knob: 1 each stage's residual on a graph branch beside its bounds
    mutable bool pdl = false;   // set while the branched step graph is captured: the main chain's
                                // launches are programmatic dependents (kbl_grid_dep_sync)
    std::string err;
    int64_t launches = 0;
    int bounds_tile = 0;        // FP32 bounds thread tile: 0 = 4x4 nodes, 1 = 4x2 nodes
    // graph of kbl_step, keyed by (w, cfl); a second slot for the other state buffer of
    // kbl_run_host_ensemble (the least recently used slot is replaced)
    cudaGraphExec_t graph = nullptr;
    double* graph_w = nullptr;
    double graph_cfl = 0.0;
    int graph_kernels = 0;
    cudaGraphExec_t graph2 = nullptr;
    double* graph2_w = nullptr;
    double graph2_cfl = 0.0;
    int graph2_kernels = 0;
    // adjoint scratch (kbl_adjoint.cu), grown on demand
    double* d_adj = nullptr;
    size_t adj_cap = 0;
    double* d_ent = nullptr;
    size_t ent_cap = 0;
};

// Frees the adjoint scratch of a context (kbl_adjoint.cu).
void kbl_adjoint_release(kbl_ctx* c);

MeshDev mesh_of(const kbl_ctx* c);

// FR operators of order p (host, FP64); defined in kbl_api.cu.
void kbl_build_fr_ops(int p, FrOps& o);
// The configuration checks of kbl_create (every entry point that takes a kbl_config applies them).
bool kbl_config_valid(const kbl_config* cfg);

// ---- launchers (kbl_fr.cu, kbl_bounds.cu, kbl_limit.cu) ------------------
// Each returns the number of kernels it launched, or -1 if the (dim, p)
// combination is not compiled in.
int launch_traces(const kbl_ctx* c, const double* w, double* wf, cudaStream_t s);
int launch_gather(const kbl_ctx* c, const double* w, const double* wf, int e0, int n,
                  double* S, cudaStream_t s);
int launch_rhs(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s);
// the FP32-mixed 2D residual with its operator products on the tensor cores (kbl_fr_tc.cu): -1 when
// not covered (order, dimension, precision, knob), -2 when these arrays cannot be TMA-mapped
int launch_rhs_tc(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s);
// folded residual operator B[K][Ns] of order p (FP64) and its split device copy (kbl_fr_tc.cu)
void kbl_rhs_operator(const FrOps& o, int p, std::vector<double>& B, int& K, int& NS);
float* kbl_rhs_tc_upload(const FrOps& o, int p);
// dt_out <- cfl * min(h / (|U| + c)); with clip, also <= t_end - t of the context
int launch_dt(const kbl_ctx* c, const double* w, double cfl, double* dt_out, int clip, cudaStream_t s);
int launch_time_advance(const kbl_ctx* c, cudaStream_t s);
// the first kernel of kbl_step: face traces of w and the clipped time step into scal[0] in one pass
int launch_traces_dt(const kbl_ctx* c, const double* w, double* wf, double cfl, cudaStream_t s);
// the time step of launch_traces_dt alone (the same dt bit for bit), for a branch beside launch_traces
int launch_dt_step(const kbl_ctx* c, const double* w, double cfl, cudaStream_t s);
// the stage kernel of kbl_step (dt from scal[0]): stage + limiter, then the next stage's traces
// (wf_next, may be nullptr) or the clock update (advance)
int launch_stage_step(const kbl_ctx* c, int stage, const double* wn, const double* ws, const double* R,
                      const double* bnd, double* wout, double* wf_next, int advance, cudaStream_t s);
int launch_bounds(const kbl_ctx* c, const double* w, const double* wf, double* bnd,
                  cudaStream_t s);
// limiting of explicit node sets U[E][ns][nv] (in place) with faces F[E][nf][nv], W[ns] host
int launch_limit_nodes(const kbl_ctx* c, int E, int ns, int nf, const double* W, double* U, const double* F,
                       const double* bnd, double* alpha, cudaStream_t s, double* F_out = nullptr,
                       const double* We = nullptr);
// Bounds of the Sec. 5 stencils of affine triangles of order p (1 or 2), gathered in the kernel
// from w[E][ns][4], wf[E][nfp][4] and the connectivity of kbl_tri (kbl_tri.cu); -1 if not covered.
int launch_bounds_tri(const kbl_ctx* c, int E, int p, const double* w, const double* wf, const int* nbr,
                      const int* nbr_edge, const double* bc, double* bnd, cudaStream_t s);
// bounds of explicit stencils S[E][nst][4] (2D, 1 <= nst <= 64); -1 for other shapes
int launch_bounds_stencil(const kbl_ctx* c, int E, int nst, const double* S, double* bnd, cudaStream_t s);
// mode 0: RK stage s fused with the limiter; mode 1: limiter only (ws = w in place)
int launch_stage(const kbl_ctx* c, int mode, int stage, const double* wn, const double* ws,
                 const double* R, const double* bnd, const double* dt, double* wout,
                 double* alpha, cudaStream_t s);

// ---- device helpers ----------------------------------------------------------
#define KBL_PI 3.14159265358979323846

// a / b: the IEEE division in FP64; in FP32 a times the special-function unit's reciprocal
// (about 1 ulp; the same reciprocal of a density is formed once and shared by every use), which
// keeps the FP32 residual off the multi-instruction IEEE division.
template <typename T>
__device__ __forceinline__ T kbl_div(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float kbl_div<float>(float a, float b) { return a * __fdividef(1.0f, b); }

template <int DIM, typename T = double>
__device__ __forceinline__ T kbl_pressure(const T* q, T gm1)
{
    T mm = q[1] * q[1];
    if (DIM == 2) mm += q[2] * q[2];
    return gm1 * (q[DIM + 1] - kbl_div(T(0.5) * mm, q[0]));
}

// Flux along axis `dir` (Eq. 2).
template <int DIM, typename T = double>
__device__ __forceinline__ void kbl_flux(const T* q, int dir, T gm1, T* F)
{
    const T P = kbl_pressure<DIM, T>(q, gm1);
    const T u = kbl_div(q[1 + dir], q[0]);
    F[0] = q[1 + dir];
    F[1] = q[1] * u + (dir == 0 ? P : T(0));
    if (DIM == 2) F[2] = q[2] * u + (dir == 1 ? P : T(0));
    F[DIM + 1] = (q[DIM + 1] + P) * u;
}

// Rusanov flux with the Davis wavespeed; ql on the minus side of the axis.
template <int DIM, typename T = double>
__device__ __forceinline__ void kbl_rusanov(const T* ql, const T* qr, int dir, T gamma, T* F)
{
    constexpr int NV = DIM + 2;
    const T gm1 = gamma - T(1);
    T Fl[NV], Fr[NV];
    kbl_flux<DIM, T>(ql, dir, gm1, Fl);
    kbl_flux<DIM, T>(qr, dir, gm1, Fr);
    const T Pl = kbl_pressure<DIM, T>(ql, gm1), Pr = kbl_pressure<DIM, T>(qr, gm1);
    const T sl = fabs(kbl_div(ql[1 + dir], ql[0])) + sqrt(kbl_div(gamma * Pl, ql[0]));
    const T sr = fabs(kbl_div(qr[1 + dir], qr[0])) + sqrt(kbl_div(gamma * Pr, qr[0]));
    const T lam = fmax(sl, sr);
#pragma unroll
    for (int v = 0; v < NV; v++) F[v] = T(0.5) * (Fl[v] + Fr[v]) - T(0.5) * lam * (qr[v] - ql[v]);
}

// HLLC flux (Toro, Spruce & Speares 1994) with the Davis wave-speed estimates
// S_l = min(U_l - c_l, U_r - c_r), S_r = max(U_l + c_l, U_r + c_r) and the contact speed S*;
// ql on the minus side of the axis.  F(ql) for 0 <= S_l, F(ql) + S_l (q*_l - ql) for
// S_l <= 0 <= S*, F(qr) + S_r (q*_r - qr) for S* <= 0 <= S_r, F(qr) for S_r <= 0, with
// q*_K = rho_K (S_K - U_K)/(S_K - S*) [1, S* along the axis, the other velocities of K,
// E_K/rho_K + (S* - U_K)(S* + P_K / (rho_K (S_K - U_K)))].
template <int DIM, typename T = double>
__device__ __forceinline__ void kbl_hllc(const T* ql, const T* qr, int dir, T gamma, T* F)
{
    constexpr int NV = DIM + 2;
    const T gm1 = gamma - T(1);
    const T Pl = kbl_pressure<DIM, T>(ql, gm1), Pr = kbl_pressure<DIM, T>(qr, gm1);
    const T Ul = kbl_div(ql[1 + dir], ql[0]), Ur = kbl_div(qr[1 + dir], qr[0]);
    const T cl = sqrt(kbl_div(gamma * Pl, ql[0])), cr = sqrt(kbl_div(gamma * Pr, qr[0]));
    const T Sl = fmin(Ul - cl, Ur - cr), Sr = fmax(Ul + cl, Ur + cr);
    const T Ss = kbl_div(Pr - Pl + ql[0] * Ul * (Sl - Ul) - qr[0] * Ur * (Sr - Ur),
                         ql[0] * (Sl - Ul) - qr[0] * (Sr - Ur));
    if (T(0) <= Sl) {
        kbl_flux<DIM, T>(ql, dir, gm1, F);
        return;
    }
    if (Sr <= T(0)) {
        kbl_flux<DIM, T>(qr, dir, gm1, F);
        return;
    }
    const bool left = Ss >= T(0);
    const T* q = left ? ql : qr;
    const T S = left ? Sl : Sr, U = left ? Ul : Ur, P = left ? Pl : Pr;
    kbl_flux<DIM, T>(q, dir, gm1, F);
    const T f = kbl_div(q[0] * (S - U), S - Ss);
    T qs[NV];
    qs[0] = f;
#pragma unroll
    for (int k = 0; k < DIM; k++) qs[1 + k] = f * (k == dir ? Ss : kbl_div(q[1 + k], q[0]));
    qs[DIM + 1] = f * (kbl_div(q[DIM + 1], q[0]) + (Ss - U) * (Ss + kbl_div(P, q[0] * (S - U))));
#pragma unroll
    for (int v = 0; v < NV; v++) F[v] += S * (qs[v] - q[v]);
}

// HLL flux (Harten, Lax & van Leer 1983; the Riemann solver of the Sedov run, Sec. 6.6)
// with the Davis estimates of kbl_hllc: F(ql) for 0 <= S_l, F(qr) for S_r <= 0, else
// (S_r F(ql) - S_l F(qr) + S_l S_r (qr - ql)) / (S_r - S_l).
template <int DIM, typename T>
__device__ __forceinline__ void kbl_hll(const T* ql, const T* qr, int dir, T gamma, T* F)
{
    constexpr int NV = DIM + 2;
    const T gm1 = gamma - T(1);
    const T Pl = kbl_pressure<DIM, T>(ql, gm1), Pr = kbl_pressure<DIM, T>(qr, gm1);
    const T Ul = kbl_div(ql[1 + dir], ql[0]), Ur = kbl_div(qr[1 + dir], qr[0]);
    const T cl = sqrt(kbl_div(gamma * Pl, ql[0])), cr = sqrt(kbl_div(gamma * Pr, qr[0]));
    const T Sl = fmin(Ul - cl, Ur - cr), Sr = fmax(Ul + cl, Ur + cr);
    if (T(0) <= Sl) {
        kbl_flux<DIM, T>(ql, dir, gm1, F);
        return;
    }
    if (Sr <= T(0)) {
        kbl_flux<DIM, T>(qr, dir, gm1, F);
        return;
    }
    T Fr[NV];
    kbl_flux<DIM, T>(ql, dir, gm1, F);
    kbl_flux<DIM, T>(qr, dir, gm1, Fr);
    const T inv = kbl_div(T(1), Sr - Sl);
#pragma unroll
    for (int v = 0; v < NV; v++) F[v] = (Sr * F[v] - Sl * Fr[v] + Sl * Sr * (qr[v] - ql[v])) * inv;
}

// Row r, component v of the wider 1D stencil of element e: the element's N solution points, then
// those of the left (face 0) and the right (face 1) neighbour; a boundary face gives its state.
template <int N>
__device__ __forceinline__ double kbl_wide1d(const double* __restrict__ w, const MeshDev& m, int e, int r, int v)
{
    const int blk = r / N, n = r - blk * N;
    if (blk == 0) return w[((size_t)v * m.E + e) * N + n];
    const int nb = m.nbr[e * 2 + (blk - 1)];
    return nb >= 0 ? w[((size_t)v * m.E + nb) * N + n] : m.bc[(size_t)(-nb - 1) * 3 + v];
}

// Exterior value of component v at face point fp of element e.
template <int DIM, int N>
__device__ __forceinline__ double kbl_exterior(const double* __restrict__ wf, const MeshDev& m,
                                               int e, int fp, int v)
{
    constexpr int NFPF = (DIM == 1) ? 1 : N;
    constexpr int NFP = (DIM == 1) ? 2 : 4 * N;
    const int f = fp / NFPF, k = fp - f * NFPF;
    const int nb = m.nbr[e * 2 * DIM + f];
    if (nb >= 0) return wf[((size_t)v * m.E + nb) * NFP + (f ^ 1) * NFPF + k];
    return m.bc[(-nb - 1) * (DIM + 2) + v];
}

template <int DIM>
__host__ __device__ constexpr int kbl_ns(int n) { return DIM == 1 ? n : n * n; }
template <int DIM>
__host__ __device__ constexpr int kbl_nfp(int n) { return DIM == 1 ? 2 : 4 * n; }

// Dispatch a templated launcher over (DIM, N = p + 1).
#define KBL_DISPATCH(DIMV, NV_, FN, ...)                                   \
    do {                                                                   \
        if ((DIMV) == 1) {                                                 \
            switch (NV_) {                                                 \
                case 2: return FN<1, 2>(__VA_ARGS__);                      \
                case 3: return FN<1, 3>(__VA_ARGS__);                      \
                case 4: return FN<1, 4>(__VA_ARGS__);                      \
                case 5: return FN<1, 5>(__VA_ARGS__);                      \
                case 6: return FN<1, 6>(__VA_ARGS__);                      \
            }                                                              \
        } else {                                                           \
            switch (NV_) {                                                 \
                case 2: return FN<2, 2>(__VA_ARGS__);                      \
                case 3: return FN<2, 3>(__VA_ARGS__);                      \
                case 4: return FN<2, 4>(__VA_ARGS__);                      \
                case 5: return FN<2, 5>(__VA_ARGS__);                      \
                case 6: return FN<2, 6>(__VA_ARGS__);                      \
            }                                                              \
        }                                                                  \
        return -1;                                                         \
    } while (0)
