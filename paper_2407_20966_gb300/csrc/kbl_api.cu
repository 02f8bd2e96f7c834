// kbl_api.cu -- host implementation of the C ABI declared in include/kbl.h.
//
// The FR operators are built here in FP64: Gauss-Legendre nodes and weights
// by the Golub-Welsch eigenvalue method (cyclic Jacobi rotations on the
// Legendre Jacobi matrix), interpolation and differentiation by the
// barycentric Lagrange formulas, and the g_DG correction derivatives from the
// nodal-DG lifting identity g_L'(x_i) = -l_i(-1) / w_i, g_R'(x_i) = l_i(1) / w_i
// that holds for Gauss-Legendre solution points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kbl_internal.cuh"

namespace {

// ---- velocity quadrature ---------------------------------------------------
// Romberg weights (units of the grid spacing h) on nu equispaced nodes, the quadrature
// Sec. 5 names beside the trapezoidal rule.  With nu - 1 = 2^L m (m odd) the rule
// extrapolates the L + 1 nested trapezoidal sums of steps 2^L h, ..., 2h, h (Richardson,
// T_k^j = T_k^(j-1) + (T_k^(j-1) - T_(k-1)^(j-1)) / (4^j - 1)).  Every sum is linear in the
// node values, so the tableau is run on weight vectors.
void romberg_weights(int nu, std::vector<double>& q)
{
    int L = 0;
    for (int m = nu - 1; m > 0 && m % 2 == 0; m /= 2) L++;
    std::vector<std::vector<double>> T(L + 1, std::vector<double>(nu, 0.0));
    for (int k = 0; k <= L; k++) {   // T[k]: trapezoidal sum of step 2^(L-k) h
        const int st = 1 << (L - k);
        for (int j = 0; j < nu; j += st) T[k][j] = (j == 0 || j == nu - 1) ? 0.5 * st : (double)st;
    }
    double f = 1.0;
    for (int lev = 1; lev <= L; lev++) {
        f *= 4.0;
        for (int k = L; k >= lev; k--)
            for (int j = 0; j < nu; j++) T[k][j] += (T[k][j] - T[k - 1][j]) / (f - 1.0);
    }
    q = T[L];
}

// ---- FR operators --------------------------------------------------------
void jacobi_eigen(int n, double* A /* n*n, symmetric, destroyed */, double* V /* n*n, columns */)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) off += A[i * n + j] * A[i * n + j];
        if (off < 1e-40) break;
        for (int p = 0; p < n; p++) {
            for (int q = p + 1; q < n; q++) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {  // A <- A J
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {  // A <- J^T A
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {  // V <- V J
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

void build_ops(int p, FrOps& o)
{
    const int n = p + 1;
    std::memset(&o, 0, sizeof(o));
    o.n = n;
    // Golub-Welsch: eigenvalues of the symmetric Jacobi matrix of the Legendre
    // recurrence are the nodes; weights are 2 * (first eigenvector entry)^2.
    double A[KBL_NMAX * KBL_NMAX] = {0}, V[KBL_NMAX * KBL_NMAX];
    for (int k = 1; k < n; k++) {
        const double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[(k - 1) * n + k] = b;
        A[k * n + (k - 1)] = b;
    }
    jacobi_eigen(n, A, V);
    int order[KBL_NMAX];
    for (int i = 0; i < n; i++) order[i] = i;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (A[order[j] * n + order[j]] < A[order[i] * n + order[i]]) std::swap(order[i], order[j]);
    for (int i = 0; i < n; i++) {
        const int k = order[i];
        o.x[i] = A[k * n + k];
        o.wq[i] = 2.0 * V[0 * n + k] * V[0 * n + k];
    }
    if (n % 2 == 1) o.x[n / 2] = 0.0;  // the middle node of an odd rule is exactly 0
    for (int i = 0; i < n / 2; i++) {   // symmetrise the rule
        const double xs = 0.5 * (o.x[n - 1 - i] - o.x[i]);
        const double ws = 0.5 * (o.wq[n - 1 - i] + o.wq[i]);
        o.x[i] = -xs; o.x[n - 1 - i] = xs;
        o.wq[i] = ws; o.wq[n - 1 - i] = ws;
    }
    // barycentric weights
    double lam[KBL_NMAX];
    for (int j = 0; j < n; j++) {
        double prod = 1.0;
        for (int m = 0; m < n; m++)
            if (m != j) prod *= (o.x[j] - o.x[m]);
        lam[j] = 1.0 / prod;
    }
    for (int side = 0; side < 2; side++) {
        const double x = side ? 1.0 : -1.0;
        double den = 0.0;
        for (int k = 0; k < n; k++) den += lam[k] / (x - o.x[k]);
        for (int j = 0; j < n; j++) {
            const double val = (lam[j] / (x - o.x[j])) / den;
            if (side) o.lp[j] = val;
            else o.lm[j] = val;
        }
    }
    for (int i = 0; i < n; i++) {
        double diag = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            o.D[i][j] = (lam[j] / lam[i]) / (o.x[i] - o.x[j]);
            diag -= o.D[i][j];
        }
        o.D[i][i] = diag;
    }
    for (int i = 0; i < n; i++) {
        o.gl[i] = -o.lm[i] / o.wq[i];
        o.gr[i] = o.lp[i] / o.wq[i];
    }
    double s1 = 0.0, s2 = 0.0, am = 0.0, ap = 0.0;
    for (int i = 0; i < n; i++) {
        s1 += o.wq[i];
        am += std::fabs(o.lm[i]);
        ap += std::fabs(o.lp[i]);
    }
    for (int k = 0; k < n * n; k++) {
        o.wm2[k] = o.wq[k % n] * o.wq[k / n];
        s2 += o.wm2[k];
    }
    o.winv1 = 1.0 / s1;
    o.winv2 = 1.0 / s2;
    o.lam = std::max(am, ap);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) o.Df[i][j] = (float)o.D[i][j];
        o.glf[i] = (float)o.gl[i];
        o.grf[i] = (float)o.gr[i];
        o.lmf[i] = (float)o.lm[i];
        o.lpf[i] = (float)o.lp[i];
        o.wqf[i] = (float)o.wq[i];
    }
    for (int k = 0; k < n * n; k++) o.wm2f[k] = (float)o.wm2[k];
    o.winv1f = (float)o.winv1;
    o.winv2f = (float)o.winv2;
    o.lamf = kbl_f32_up(o.lam);
}

kbl_status fail(kbl_ctx* c, kbl_status st, const char* msg)
{
    if (c) c->err = msg;
    return st;
}

kbl_status cuda_fail(kbl_ctx* c, cudaError_t e, const char* where)
{
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return KBL_ECUDA;
}

// Post-launch check of a launcher result.
kbl_status after_launch(kbl_ctx* c, int n, const char* where)
{
    if (n < 0) return fail(c, KBL_EINVAL, "order/dimension not compiled in");
    c->launches += n;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return KBL_OK;
}

void drop_graphs(kbl_ctx* c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph2) cudaGraphExecDestroy(c->graph2);
    c->graph = c->graph2 = nullptr;
    c->graph_w = c->graph2_w = nullptr;
}

void free_mesh(kbl_ctx* c)
{
    double** bufs[] = {&c->d_h, &c->d_bc, &c->d_wf, &c->d_R, &c->d_bnd, &c->d_wa, &c->d_wb, &c->d_whost, &c->d_whost2};
    for (double** b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    if (c->d_nbr) cudaFree(c->d_nbr);
    c->d_nbr = nullptr;
    kbl_adjoint_release(c);
    drop_graphs(c);
    c->mesh_ready = false;
}

bool ready(kbl_ctx* c) { return c && c->mesh_ready; }

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

// Issue one full SSP-RK3 step on stream s (for capture): the traces and the clipped time step of w,
// then per stage the residual, the bounds and the stage + limiter kernel, which also writes the
// next stage's traces (stages 0 and 1) or advances the clock (stage 2).  Without a side stream:
// 10 ordinary launches in one chain (traces and time step in one kernel).  With a side stream s2
// and its events (ctx->pdl set): the time step runs on the side branch beside the traces, and the
// main chain's kernels (traces, residual, bounds, stage) are programmatic dependents, each
// waiting for its predecessor before it touches memory and letting its own dependent launch at
// once; the stage kernel waits only before it reads the bounds (kbl_limit_body.cuh), so its
// combination and screen overlap the bounds launch's last blocks: 11 kernels.  A residual on a
// branch beside the bounds measured no better than in the chain: the bounds kernel holds the
// issue slots and the residency either way.
int issue_step(kbl_ctx* c, double* w, double cfl, cudaStream_t s, cudaStream_t s2 = nullptr,
               cudaEvent_t* ev = nullptr)
{
    int n = 0, r;
    if (s2) {
        // the time step on the side branch, beside the traces: only the stage kernels read it, and
        // they run after the branch joins (the first residual follows it on the same stream)
        if (cudaEventRecord(ev[6], s) != cudaSuccess || cudaStreamWaitEvent(s2, ev[6], 0) != cudaSuccess) return -1;
        if ((r = launch_dt_step(c, w, cfl, s2)) < 0) return -1;
        n += r;
        if ((r = launch_traces(c, w, c->d_wf, s)) < 0) return -1;
        n += r;
    } else {
        if ((r = launch_traces_dt(c, w, c->d_wf, cfl, s)) < 0) return -1;
        n += r;
    }
    const double* wn = w;
    const double* ws = w;
    double* outs[3] = {c->d_wa, c->d_wb, w};
    // with a side stream the main chain is residual -> bounds -> stage per stage, each a
    // programmatic dependent of the one before; the time step (side branch) joins before the
    // first residual
    if (s2 && cudaEventRecord(ev[0], s2) != cudaSuccess) return -1;
    for (int st = 0; st < 3; st++) {
        if (s2 && st == 0 && cudaStreamWaitEvent(s, ev[0], 0) != cudaSuccess) return -1;
        if ((r = launch_rhs(c, ws, c->d_wf, c->d_R, s)) < 0) return -1;
        n += r;
        if ((r = launch_bounds(c, ws, c->d_wf, c->d_bnd, s)) < 0) return -1;
        n += r;
        if ((r = launch_stage_step(c, st, wn, ws, c->d_R, c->d_bnd, outs[st], st < 2 ? c->d_wf : nullptr, st == 2, s)) <
            0)
            return -1;
        n += r;
        ws = outs[st];
    }
    return n;
}

}  // namespace

void kbl_build_fr_ops(int p, FrOps& o) { build_ops(p, o); }

bool kbl_config_valid(const kbl_config* cfg)
{
    if (!cfg) return false;
    if (cfg->dim != 1 && cfg->dim != 2) return false;
    if (cfg->p < 1 || cfg->p > KBL_PMAX) return false;
    if (cfg->dim == 2) {
        const int nx = cfg->nu[0];
        if (cfg->nu[1] != nx || nx < 2 || nx > 64) return false;
    } else if (cfg->nu[0] < 2 || cfg->nu[0] > 4096) {
        return false;
    }
    if (!(cfg->gamma > 1.0) || !(cfg->k > 0.0) || !(cfg->r_fac >= 0.0 && cfg->r_fac < 1.0) ||
        !(cfg->eps >= 0.0) || !(cfg->rho_floor >= 0.0) || !(cfg->p_floor >= 0.0))
        return false;
    if (cfg->eps_rule != 0 && cfg->eps_rule != 1) return false;
    if (cfg->stencil != 0 && !(cfg->stencil == 1 && cfg->dim == 1)) return false;
    if (cfg->precision != KBL_FP64 && cfg->precision != KBL_FP32_MIXED) return false;
    if (cfg->uncoupled != 0 && cfg->uncoupled != 1) return false;
    if (cfg->flux < 0 || cfg->flux > 2) return false;
    if (cfg->quadrature != 0 && cfg->quadrature != 1) return false;
    if (cfg->quadrature == 1 && (cfg->nu[0] < 3 || (cfg->nu[0] - 1) % 2 != 0)) return false;
    return true;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

kbl_status kbl_config_default(kbl_config* cfg, int dim, int p)
{
    if (!cfg || (dim != 1 && dim != 2) || p < 1 || p > KBL_PMAX) return KBL_EINVAL;
    cfg->dim = dim;
    cfg->p = p;
    cfg->nu[0] = dim == 1 ? 64 : 32;
    cfg->nu[1] = dim == 1 ? 1 : 32;
    cfg->gamma = 1.4;
    cfg->k = 4.0;
    cfg->r_fac = 1e-3;
    cfg->eps = 1e-13;
    cfg->rho_floor = 1e-12;
    cfg->p_floor = 1e-12;
    cfg->eps_rule = 0;
    cfg->precision = KBL_FP64;
    cfg->uncoupled = 0;
    cfg->flux = 0;
    cfg->quadrature = 0;
    cfg->stencil = 0;
    return KBL_OK;
}

kbl_status kbl_create(kbl_ctx** out, const kbl_config* cfg, void* cuda_stream)
{
    if (!out) return KBL_EINVAL;
    *out = nullptr;
    if (!kbl_config_valid(cfg)) return KBL_EINVAL;
    kbl_ctx* c = new (std::nothrow) kbl_ctx();
    if (!c) return KBL_ENOMEM;
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->phys.gamma = cfg->gamma;
    c->phys.k = cfg->k;
    c->phys.r_fac = cfg->r_fac;
    c->phys.eps = cfg->eps;
    c->phys.rho_floor = cfg->rho_floor;
    c->phys.p_floor = cfg->p_floor;
    c->phys.eps_rule = cfg->eps_rule;
    c->phys.nu[0] = cfg->nu[0];
    c->phys.nu[1] = cfg->dim == 2 ? cfg->nu[1] : 1;
    c->phys.uncoupled = cfg->uncoupled;
    c->phys.flux = cfg->flux;
    c->phys.qw = nullptr;
    c->phys.qwf = nullptr;
    kbl_phys_derive(c->phys);
    build_ops(cfg->p, c->ops);
    const int n = cfg->p + 1;
    c->nv = cfg->dim + 2;
    c->ns = cfg->dim == 1 ? n : n * n;
    c->nfp = cfg->dim == 1 ? 2 : 4 * n;
    c->nsten = cfg->stencil == 1 ? 3 * c->ns : c->ns + 2 * c->nfp;
    cudaError_t e;
    if ((e = dalloc(&c->d_scal, 4)) != cudaSuccess || (e = dalloc(&c->d_dtbits, 1)) != cudaSuccess ||
        (e = dalloc(&c->d_blocks_done, 1)) != cudaSuccess ||
        (e = dalloc(&c->d_flags, 1)) != cudaSuccess) {
        kbl_destroy(c);
        return KBL_ECUDA;
    }
    if (cfg->quadrature == 1) {
        // the table in FP64, then its FP32 copy, in one allocation
        const int nq = cfg->nu[0];
        std::vector<double> q;
        romberg_weights(nq, q);
        std::vector<double> buf(nq + (nq + 1) / 2, 0.0);
        std::copy(q.begin(), q.end(), buf.begin());
        float* qf = reinterpret_cast<float*>(buf.data() + nq);
        for (int j = 0; j < nq; j++) qf[j] = (float)q[j];
        if ((e = dalloc(&c->d_qw, buf.size())) != cudaSuccess ||
            (e = cudaMemcpy(c->d_qw, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
            kbl_destroy(c);
            return KBL_ECUDA;
        }
        c->phys.qw = c->d_qw;
        c->phys.qwf = reinterpret_cast<const float*>(c->d_qw + nq);
    }
    if (cfg->dim == 2 && cfg->precision == KBL_FP32_MIXED) c->d_tcop = kbl_rhs_tc_upload(c->ops, cfg->p);
    const double scal[4] = {0.0, 0.0, INFINITY, 0.0};
    if ((e = cudaMemcpy(c->d_scal, scal, sizeof(scal), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c->d_dtbits, 0x7f, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(c->d_blocks_done, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(c->d_flags, 0, sizeof(DevFlags))) != cudaSuccess) {
        kbl_destroy(c);
        return KBL_ECUDA;
    }
    *out = c;
    return KBL_OK;
}

kbl_status kbl_residual_operator(int p, double* host_out, int n)
{
    if (!host_out || p < 1 || p > KBL_PMAX) return KBL_EINVAL;
    FrOps o;
    build_ops(p, o);
    std::vector<double> B;
    int K = 0, NS = 0;
    kbl_rhs_operator(o, p, B, K, NS);
    if (n < K * NS) return KBL_EINVAL;
    std::copy(B.begin(), B.end(), host_out);
    return KBL_OK;
}

kbl_status kbl_velocity_weights(int nu, int quadrature, double* host_out)
{
    if (!host_out || nu < 2 || (quadrature != 0 && quadrature != 1)) return KBL_EINVAL;
    if (quadrature == 1) {
        if ((nu - 1) % 2 != 0) return KBL_EINVAL;
        std::vector<double> q;
        romberg_weights(nu, q);
        std::copy(q.begin(), q.end(), host_out);
    } else {
        for (int j = 0; j < nu; j++) host_out[j] = (j == 0 || j == nu - 1) ? 0.5 : 1.0;
    }
    return KBL_OK;
}

kbl_status kbl_destroy(kbl_ctx* c)
{
    if (!c) return KBL_EINVAL;
    free_mesh(c);
    if (c->d_scal) cudaFree(c->d_scal);
    if (c->d_dtbits) cudaFree(c->d_dtbits);
    if (c->d_blocks_done) cudaFree(c->d_blocks_done);
    if (c->d_flags) cudaFree(c->d_flags);
    if (c->d_qw) cudaFree(c->d_qw);
    if (c->d_tcop) cudaFree(c->d_tcop);
    if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
    if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
    for (int k = 0; k < 2; k++) {
        if (c->ev_h2d[k]) cudaEventDestroy(c->ev_h2d[k]);
        if (c->ev_step[k]) cudaEventDestroy(c->ev_step[k]);
        if (c->ev_d2h[k]) cudaEventDestroy(c->ev_d2h[k]);
    }
    delete c;
    return KBL_OK;
}

kbl_status kbl_set_stream(kbl_ctx* c, void* s)
{
    if (!c) return KBL_EINVAL;
    c->stream = (cudaStream_t)s;
    return KBL_OK;
}

const char* kbl_last_error(const kbl_ctx* c) { return c ? c->err.c_str() : "null context"; }
int kbl_nv(const kbl_ctx* c) { return c ? c->nv : -1; }
int kbl_ns(const kbl_ctx* c) { return c ? c->ns : -1; }
int kbl_nfp(const kbl_ctx* c) { return c ? c->nfp : -1; }
int kbl_nstencil(const kbl_ctx* c) { return c ? c->nsten : -1; }
int64_t kbl_launch_count(const kbl_ctx* c) { return c ? c->launches : -1; }

kbl_status kbl_mesh_upload(kbl_ctx* c, int n_elem, const int32_t* nbr, const double* h, int n_bc,
                           const double* bc)
{
    if (!c) return KBL_EINVAL;
    const int d = c->cfg.dim, nv = c->nv;
    if (n_elem < 0 || n_bc < 0) return fail(c, KBL_EINVAL, "negative size");
    if (n_elem > 0 && (!nbr || !h)) return fail(c, KBL_EINVAL, "null mesh array");
    if (n_bc > 0 && !bc) return fail(c, KBL_EINVAL, "null boundary states");
    for (long i = 0; i < (long)n_elem * 2 * d; i++) {
        const int b = nbr[i];
        if (b >= n_elem || (b < 0 && -(b + 1) >= n_bc))
            return fail(c, KBL_EINVAL, "neighbour index or boundary id out of range");
    }
    for (long i = 0; i < (long)n_elem * d; i++)
        if (!(h[i] > 0.0)) return fail(c, KBL_EINVAL, "element width must be positive");
    cudaStreamSynchronize(c->stream);
    free_mesh(c);
    c->E = n_elem;
    c->n_bc = n_bc;
    const size_t E = (size_t)n_elem;
    cudaError_t e;
    if ((e = dalloc(&c->d_nbr, E * 2 * d)) != cudaSuccess || (e = dalloc(&c->d_h, E * d)) != cudaSuccess ||
        (e = dalloc(&c->d_bc, (size_t)n_bc * nv)) != cudaSuccess ||
        (e = dalloc(&c->d_wf, E * nv * c->nfp)) != cudaSuccess ||
        (e = dalloc(&c->d_R, E * nv * c->ns)) != cudaSuccess ||
        (e = dalloc(&c->d_bnd, E * nv * 2)) != cudaSuccess ||
        (e = dalloc(&c->d_wa, E * nv * c->ns)) != cudaSuccess ||
        (e = dalloc(&c->d_wb, E * nv * c->ns)) != cudaSuccess ||
        (e = dalloc(&c->d_whost, E * nv * c->ns)) != cudaSuccess) {
        free_mesh(c);
        c->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? KBL_ENOMEM : KBL_ECUDA;
    }
    if (n_elem > 0) {
        if ((e = cudaMemcpy(c->d_nbr, nbr, E * 2 * d * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(c->d_h, h, E * d * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_mesh(c);
            return cuda_fail(c, e, "mesh copy");
        }
    }
    if (n_bc > 0 && (e = cudaMemcpy(c->d_bc, bc, (size_t)n_bc * nv * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_mesh(c);
        return cuda_fail(c, e, "boundary copy");
    }
    c->mesh_ready = true;
    return KBL_OK;
}

kbl_status kbl_get_operator(const kbl_ctx* c, int which, double* out, int n)
{
    if (!c || !out) return KBL_EINVAL;
    const int np = c->ops.n;
    const int need = (which == 4) ? np * np : np;
    if (which < 0 || which > 6 || n < need) return KBL_EINVAL;
    for (int i = 0; i < np; i++) {
        switch (which) {
            case 0: out[i] = c->ops.x[i]; break;
            case 1: out[i] = c->ops.wq[i]; break;
            case 2: out[i] = c->ops.lm[i]; break;
            case 3: out[i] = c->ops.lp[i]; break;
            case 4: for (int m = 0; m < np; m++) out[i * np + m] = c->ops.D[i][m]; break;
            case 5: out[i] = c->ops.gl[i]; break;
            case 6: out[i] = c->ops.gr[i]; break;
        }
    }
    return KBL_OK;
}

kbl_status kbl_traces(kbl_ctx* c, const double* w, double* wf)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (c->E > 0 && (!w || !wf)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_traces(c, w, wf, c->stream), "traces");
}

kbl_status kbl_gather_stencil(kbl_ctx* c, const double* w, const double* wf, int e0, int n, double* S)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (e0 < 0 || n < 0 || (long)e0 + n > c->E) return fail(c, KBL_EINVAL, "element range");
    if (n > 0 && (!w || !wf || !S)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_gather(c, w, wf, e0, n, S, c->stream), "gather");
}

kbl_status kbl_bounds(kbl_ctx* c, const double* w, const double* wf, double* bnd)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (c->E > 0 && (!w || !wf || !bnd)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_bounds(c, w, wf, bnd, c->stream), "bounds");
}

kbl_status kbl_bounds_stencil(kbl_ctx* c, int n_elem, int n_states, const double* S, double* bnd)
{
    if (!c) return KBL_EINVAL;
    if (c->cfg.dim != 2) return fail(c, KBL_EINVAL, "explicit stencils are 2D");
    if (n_elem < 0 || n_states < 1 || n_states > 64) return fail(c, KBL_EINVAL, "n_elem >= 0, 1 <= n_states <= 64");
    if (n_elem > 0 && (!S || !bnd)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_bounds_stencil(c, n_elem, n_states, S, bnd, c->stream), "bounds_stencil");
}

kbl_status kbl_limit_nodes(kbl_ctx* c, int n_elem, int ns, int nf, const double* W, double* U, const double* F,
                           const double* bnd, double* alpha)
{
    if (!c) return KBL_EINVAL;
    if (n_elem < 0 || ns < 1 || ns > 64 || nf < 0 || nf > 64) return fail(c, KBL_EINVAL, "1 <= ns <= 64, 0 <= nf <= 64");
    if (!W) return fail(c, KBL_EINVAL, "null weights");
    for (int n = 0; n < ns; n++)
        if (!(W[n] > 0.0) || !(W[n] < INFINITY)) return fail(c, KBL_EINVAL, "mean weights must be positive");
    if (n_elem > 0 && (!U || !bnd || (nf > 0 && !F))) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_limit_nodes(c, n_elem, ns, nf, W, U, F, bnd, alpha, c->stream), "limit_nodes");
}

kbl_status kbl_rhs(kbl_ctx* c, const double* w, const double* wf, double* R)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (c->E > 0 && (!w || !wf || !R)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_rhs(c, w, wf, R, c->stream), "rhs");
}

kbl_status kbl_limit(kbl_ctx* c, double* w, const double* bnd, double* alpha)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (c->E > 0 && (!w || !bnd)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_stage(c, 1, 0, w, w, nullptr, bnd, nullptr, w, alpha, c->stream), "limit");
}

kbl_status kbl_stage(kbl_ctx* c, int s, const double* wn, const double* ws, const double* R,
                     const double* bnd, const double* dt_dev, double* wout, double* alpha)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (s < 0 || s > 2) return fail(c, KBL_EINVAL, "stage must be 0, 1 or 2");
    if (c->E > 0 && (!wn || !ws || !R || !bnd || !dt_dev || !wout)) return fail(c, KBL_EINVAL, "null array");
    return after_launch(c, launch_stage(c, 0, s, wn, ws, R, bnd, dt_dev, wout, alpha, c->stream), "stage");
}

kbl_status kbl_dt(kbl_ctx* c, const double* w, double cfl, double* dt_dev)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (!dt_dev || (c->E > 0 && !w) || !(cfl > 0.0)) return fail(c, KBL_EINVAL, "bad argument");
    // the context's end time is not applied here: dt_dev gets cfl * min(h / (|U| + c))
    return after_launch(c, launch_dt(c, w, cfl, dt_dev, 0, c->stream), "dt");
}

kbl_status kbl_set_time(kbl_ctx* c, double t, double t_end)
{
    if (!c) return KBL_EINVAL;
    const double v[2] = {t, t_end};
    cudaError_t e = cudaMemcpyAsync(c->d_scal + 1, v, sizeof(v), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_time");
    return KBL_OK;
}

kbl_status kbl_time_sync(kbl_ctx* c, double* t)
{
    if (!c || !t) return KBL_EINVAL;
    cudaError_t e = cudaMemcpyAsync(t, c->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "time_sync");
    return KBL_OK;
}

kbl_status kbl_step(kbl_ctx* c, double* w, double cfl)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if ((c->E > 0 && !w) || !(cfl > 0.0)) return fail(c, KBL_EINVAL, "bad argument");
    if (c->E == 0) return KBL_OK;
    if (c->graph2 && c->graph2_w == w && c->graph2_cfl == cfl) {   // most recently used slot first
        std::swap(c->graph, c->graph2);
        std::swap(c->graph_w, c->graph2_w);
        std::swap(c->graph_cfl, c->graph2_cfl);
        std::swap(c->graph_kernels, c->graph2_kernels);
    }
    if (!(c->graph && c->graph_w == w && c->graph_cfl == cfl)) {
        // the new graph takes the first slot; the previous one moves to the second
        if (c->graph2) cudaGraphExecDestroy(c->graph2);
        c->graph2 = c->graph;
        c->graph2_w = c->graph_w;
        c->graph2_cfl = c->graph_cfl;
        c->graph2_kernels = c->graph_kernels;
        c->graph = nullptr;
        c->graph_w = nullptr;
        cudaStream_t cap = nullptr, side = nullptr;
        cudaEvent_t ev[7] = {};
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        // the side branch (the time step, beside the first traces) at the highest priority, so
        // that its blocks are placed before the traces kernel's later blocks
        int prio_lo = 0, prio_hi = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (e == cudaSuccess && c->overlap_rhs)
            e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_hi);
        for (int k = 0; k < 7 && e == cudaSuccess && side; k++)
            e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        auto release = [&]() {
            for (int k = 0; k < 7; k++)
                if (ev[k]) cudaEventDestroy(ev[k]);
            if (side) cudaStreamDestroy(side);
            if (cap) cudaStreamDestroy(cap);
        };
        if (e != cudaSuccess) {
            release();
            return cuda_fail(c, e, "capture stream");
        }
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(c, e, "begin capture");
        }
        c->pdl = side != nullptr;   // the main chain of the branched graph as programmatic dependents
        const int n = issue_step(c, w, cfl, cap, side, ev);
        c->pdl = false;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        release();
        if (n < 0) {
            if (g) cudaGraphDestroy(g);
            return fail(c, KBL_EINVAL, "order/dimension not compiled in");
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            return cuda_fail(c, e, "instantiate");
        }
        c->graph_w = w;
        c->graph_cfl = cfl;
        c->graph_kernels = n;
    }
    cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    c->launches += c->graph_kernels;
    return KBL_OK;
}

kbl_status kbl_run_host(kbl_ctx* c, const double* win, double* wout, int n_steps, double cfl)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (n_steps < 0 || !(cfl > 0.0) || (c->E > 0 && (!win || !wout))) return fail(c, KBL_EINVAL, "bad argument");
    const size_t bytes = (size_t)c->E * c->nv * c->ns * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(c->d_whost, win, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "H2D");
    for (int i = 0; i < n_steps; i++) {
        kbl_status st = kbl_step(c, c->d_whost, cfl);
        if (st != KBL_OK) return st;
    }
    e = cudaMemcpyAsync(wout, c->d_whost, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "D2H");
    return KBL_OK;
}

kbl_status kbl_run_host_ensemble(kbl_ctx* c, int n_members, const double* win, double* wout, int n_steps,
                                 double cfl)
{
    if (!ready(c)) return fail(c, KBL_ESTATE, "no mesh");
    if (n_members < 0 || n_steps < 0 || !(cfl > 0.0) || (c->E > 0 && n_members > 0 && (!win || !wout)))
        return fail(c, KBL_EINVAL, "bad argument");
    if (c->E == 0 || n_members == 0) return KBL_OK;
    const size_t count = (size_t)c->E * c->nv * c->ns;
    cudaError_t e = cudaSuccess;
    if (!c->d_whost2) e = dalloc(&c->d_whost2, count);
    if (e == cudaSuccess && !c->s_h2d) e = cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->s_d2h) e = cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        if (!c->ev_h2d[k]) e = cudaEventCreateWithFlags(&c->ev_h2d[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !c->ev_step[k]) e = cudaEventCreateWithFlags(&c->ev_step[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !c->ev_d2h[k]) e = cudaEventCreateWithFlags(&c->ev_d2h[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "ensemble set-up");
    double* buf[2] = {c->d_whost, c->d_whost2};
    // every member starts from the context's current time: keep it in scal[3]; the copies wait
    // for the work queued on the context's stream before this call
    e = cudaMemcpyAsync(c->d_scal + 3, c->d_scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_step[1], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_h2d, c->ev_step[1], 0);
    for (int k = 0; k < n_members && e == cudaSuccess; k++) {
        const int b = k & 1;
        const double* in = win + (size_t)k * count;
        double* out = wout + (size_t)k * count;
        if (k >= 2) e = cudaStreamWaitEvent(c->s_h2d, c->ev_d2h[b], 0);   // member k-2 has left buf[b]
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf[b], in, count * sizeof(double), cudaMemcpyHostToDevice, c->s_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_h2d[b], c->s_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_h2d[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_scal + 1, c->d_scal + 3, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) break;
        for (int i = 0; i < n_steps; i++) {
            const kbl_status st = kbl_step(c, buf[b], cfl);
            if (st != KBL_OK) {
                cudaStreamSynchronize(c->s_h2d);
                cudaStreamSynchronize(c->s_d2h);
                return st;
            }
        }
        e = cudaEventRecord(c->ev_step[b], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_d2h, c->ev_step[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf[b], count * sizeof(double), cudaMemcpyDeviceToHost, c->s_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_d2h[b], c->s_d2h);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_h2d);
    if (e != cudaSuccess) return cuda_fail(c, e, "ensemble run");
    return KBL_OK;
}

kbl_status kbl_read_counters(kbl_ctx* c, kbl_counters* out)
{
    if (!c || !out) return KBL_EINVAL;
    DevFlags f;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&f, c->d_flags, sizeof(f), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_flags, 0, sizeof(DevFlags));
    if (e != cudaSuccess) return cuda_fail(c, e, "counters");
    out->nonphysical = f.nonphysical;
    out->timeout = f.timeout;
    out->limited_elements = (int64_t)f.limited;
    out->pressure_relimits = (int64_t)f.prelimit;
    out->eps_rule_activations = (int64_t)f.eps_rule;
    out->mean_outside_bounds = (int64_t)f.mean_outside;
    for (int k = 0; k < KBL_ALPHA_BINS; k++) out->alpha_hist[k] = (int64_t)f.alpha_hist[k];
    if (f.timeout) return fail(c, KBL_ETIMEOUT, "a bounded device wait gave up");
    if (f.nonphysical) return fail(c, KBL_ENONPHYSICAL, "non-physical stencil state (rho <= 0 or P <= 0)");
    return KBL_OK;
}

kbl_status kbl_set_tuning(kbl_ctx* c, int key, int value)
{
    if (!c) return KBL_EINVAL;
    if (key == KBL_TUNE_RHS_TC && (value == 0 || value == 1)) {
        c->rhs_tc = value;
        drop_graphs(c);
        return KBL_OK;
    }
    if (key == KBL_TUNE_RHS_OVERLAP && (value == 0 || value == 1)) {
        c->overlap_rhs = value;
        drop_graphs(c);
        return KBL_OK;
    }
    if (key != KBL_TUNE_BOUNDS_TILE || value < 0 || value > 2) return fail(c, KBL_EINVAL, "unknown tuning knob or value");
    c->bounds_tile = value;
    drop_graphs(c);
    return KBL_OK;
}

kbl_status kbl_get_tuning(const kbl_ctx* c, int key, int* value)
{
    if (!c || !value) return KBL_EINVAL;
    if (key == KBL_TUNE_BOUNDS_TILE) *value = c->bounds_tile;
    else if (key == KBL_TUNE_RHS_TC) *value = c->rhs_tc;
    else if (key == KBL_TUNE_RHS_OVERLAP) *value = c->overlap_rhs;
    else return KBL_EINVAL;
    return KBL_OK;
}

kbl_status kbl_check(kbl_ctx* c)
{
    kbl_counters k;
    return kbl_read_counters(c, &k);
}

}  // extern "C"
